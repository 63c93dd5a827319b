// Block- and warp-level device functions of libtga, shared by the
// single-instance kernels (tga_kernels.cu), the persistent single-instance
// descent (tga_persist.cu) and the persistent batched kernel (tga_batch.cu).
//
// TGA_LDG(p) loads data that the search mutates (positions, attribute
// records, the position-ordered distance copy).  The per-step kernels define
// it as __ldg: their state changes only between launches.  The persistent
// kernels, where several SMs read state that another SM rewrote during the
// same launch, define it as a plain load and are compiled with L1 caching of
// global loads disabled (-dlcm=cg), so every such read is served by L2.
//
// Template flag PD (pickups, the VRPSPDTW; always with time windows): the
// load term of a route is that of its largest load on board, evaluated from
// the incoming / outgoing / largest loads of Section 4.3.2.  Without it the
// code is the CVRP / VRPTW one, where loads simply add.
#pragma once
#ifndef TGA_LDG
#error "define TGA_LDG before including tga_device.cuh"
#endif

#include "tga_internal.cuh"
#undef TGA_FILE_ID
#define TGA_FILE_ID 2

namespace tga {
// internal linkage: each translation unit compiles these with its own TGA_LDG
namespace {


// ---------------------------------------------------------------------------
// helpers

__device__ __forceinline__ void set_status(Control *C, int code) {
    atomicCAS(&C->status, 0, code);
}

// GPU-scope release/acquire operations (PTX memory model) for the hand-offs
// between CTAs: lighter than a sequentially consistent fence around a
// relaxed atomic.  A release by thread 0 after __syncthreads publishes the
// whole block's earlier writes; an acquire by thread 0 followed by
// __syncthreads orders the whole block's later reads.
__device__ __forceinline__ int atom_add_acq_rel(int *p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void red_add_release(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ Seg shfl_seg_up(const Seg &s, int off) {
    Seg o;
    o.E = __shfl_up_sync(0xffffffffu, s.E, off);
    o.L = __shfl_up_sync(0xffffffffu, s.L, off);
    o.D = __shfl_up_sync(0xffffffffu, s.D, off);
    o.TW = __shfl_up_sync(0xffffffffu, s.TW, off);
    o.dist = __shfl_up_sync(0xffffffffu, s.dist, off);
    o.load = __shfl_up_sync(0xffffffffu, s.load, off);
    o.out = __shfl_up_sync(0xffffffffu, s.out, off);
    return o;
}

__device__ __forceinline__ Seg shfl_seg_down(const Seg &s, int off) {
    Seg o;
    o.E = __shfl_down_sync(0xffffffffu, s.E, off);
    o.L = __shfl_down_sync(0xffffffffu, s.L, off);
    o.D = __shfl_down_sync(0xffffffffu, s.D, off);
    o.TW = __shfl_down_sync(0xffffffffu, s.TW, off);
    o.dist = __shfl_down_sync(0xffffffffu, s.dist, off);
    o.load = __shfl_down_sync(0xffffffffu, s.load, off);
    o.out = __shfl_down_sync(0xffffffffu, s.out, off);
    return o;
}

__device__ __forceinline__ Seg shfl_seg_idx(const Seg &s, int src) {
    Seg o;
    o.E = __shfl_sync(0xffffffffu, s.E, src);
    o.L = __shfl_sync(0xffffffffu, s.L, src);
    o.D = __shfl_sync(0xffffffffu, s.D, src);
    o.TW = __shfl_sync(0xffffffffu, s.TW, src);
    o.dist = __shfl_sync(0xffffffffu, s.dist, src);
    o.load = __shfl_sync(0xffffffffu, s.load, src);
    o.out = __shfl_sync(0xffffffffu, s.out, src);
    return o;
}

__device__ __forceinline__ Ld shfl_ld_up(const Ld &s, int off) {
    Ld o;
    o.i = __shfl_up_sync(0xffffffffu, s.i, off);
    o.o = __shfl_up_sync(0xffffffffu, s.o, off);
    o.m = __shfl_up_sync(0xffffffffu, s.m, off);
    return o;
}

__device__ __forceinline__ Ld shfl_ld_down(const Ld &s, int off) {
    Ld o;
    o.i = __shfl_down_sync(0xffffffffu, s.i, off);
    o.o = __shfl_down_sync(0xffffffffu, s.o, off);
    o.m = __shfl_down_sync(0xffffffffu, s.m, off);
    return o;
}

__device__ __forceinline__ Ld shfl_ld_idx(const Ld &s, int src) {
    Ld o;
    o.i = __shfl_sync(0xffffffffu, s.i, src);
    o.o = __shfl_sync(0xffffffffu, s.o, src);
    o.m = __shfl_sync(0xffffffffu, s.m, src);
    return o;
}

__device__ __forceinline__ int route_node(const Dev &d, int start, int L, int k) {
    return (k <= 0 || k > L) ? 0 : d.seq[TGA_IX(start + k, d.Wp)];
}

__device__ __forceinline__ int route_anchor(const Dev &d, int r, int start, int L, int k) {
    return k == 0 ? d.n + 1 + r : route_node(d, start, L, k);
}

// Constants of the swaps of runs for the customer x at index k >= 1 of a
// route (XRec): p* = the predecessor's prefix (distance, warp, departure),
// g* = x's suffix after it, g1* = the suffix after x+ (has1: x+ is a
// customer), run = the segment x, x+ (valid when has1), d1 = x+'s demand.
__device__ __forceinline__ XRec make_xrec(int wTe, int Rcost, int Rload, int Q, int pdist, int ptwf, int ptau,
                                          int gdist, int gtw, int gL, bool has1, int g1dist, int g1tw, int g1L,
                                          const Seg &run, int d1, int e, int l, int sv, int dx) {
    XRec x;
    x.S1 = pdist + gdist + wTe * (ptwf + gtw) - Rcost;
    x.tauP = ptau; x.Lg1 = gL; x.LQd1 = Rload - dx - Q;
    if (has1) {
        x.S2 = pdist + g1dist + wTe * (ptwf + g1tw) - Rcost;
        x.Lg2 = g1L; x.LQd2 = Rload - dx - d1 - Q; x.ld2 = dx + d1;
        x.E2 = run.E; x.L2 = run.L; x.Dm2 = run.D - run.TW; x.RC2 = run.dist + wTe * run.TW;
    } else {
        x.S2 = kBig; x.Lg2 = 0; x.LQd2 = 0; x.ld2 = 0; x.E2 = 0; x.L2 = 0; x.Dm2 = 0; x.RC2 = 0;
    }
    x.e = e; x.l = l; x.s = sv; x.d = dx;
    return x;
}

__device__ __forceinline__ XRec xrec_none() {
    XRec x{};
    x.S1 = kBig; x.S2 = kBig;
    return x;
}

// Rebuild every attribute of route r with one warp (all 32 lanes must call).
// Elements of the route: 0 = start depot, 1..L customers, L+1 = end depot.
// Forward inclusive scan gives the prefix F(x) of every anchor, backward
// inclusive scan the suffix; the route's totals are the prefix of the end
// depot.  Routes longer than 32 elements are scanned in chunks with a carry.
// PD (pickups): the loads L_I, L_O, L_M (Section 4.3.2) are scanned beside.
// XS: also the constants of the swaps of runs (XRec).
template <bool PD, bool XS = false>
__device__ void rebuild_route(const Dev &d, int r, int lane) {
    const RouteRec rr = d.rrec[TGA_IX(r, d.m)];
    const int st = rr.start, L = rr.len, E = L + 2;
    const bool tw = d.has_tw != 0;
    constexpr bool pd = PD;
    const int wTe = tw ? d.wT : 0;
    // ---- forward scan: prefixes
    Seg carry{};
    Ld lcarry{0, 0, 0};
    bool have = false;
    for (int base = 0; base < E; base += 32) {
        const int k = base + lane;
        const bool valid = k < E;
        const int x = valid ? route_node(d, st, L, k) : 0;
        const int nx = (k + 1 < E) ? route_node(d, st, L, k + 1) : 0;
        const int out = (valid && k + 1 < E) ? dmat(d, x, nx) : 0;
        Seg s = seg_node(d, x, out);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            Seg o = shfl_seg_up(s, off);
            if (lane >= off) s = seg_cat(o, s);
        }
        if (have) s = seg_cat(carry, s);
        Ld l{0, 0, 0};
        if (pd) {
            l = ld_node(d, x);
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const Ld o = shfl_ld_up(l, off);
                if (lane >= off) l = ld_cat(o, l);
            }
            if (have) l = ld_cat(lcarry, l);
        }
        if (valid) {
            if (k <= L) {
                const int a = route_anchor(d, r, st, L, k);
                BRec *b = d.brec + TGA_IX(a, d.W + 1);
                b->node = x; b->route = r; b->idx = k;
                b->tau = tw ? s.E + s.D - s.TW : 0;
                b->twf = tw ? s.TW : 0;
                b->distf = s.dist;
                b->loadf = s.load;
                if (pd) { b->lof = l.o; b->lmf = l.m; }
            } else {
                RouteRec *R = d.rrec + TGA_IX(r, d.m);
                const int twr = tw ? s.TW : 0;
                const int lm = pd ? l.m : s.load;
                R->load = s.load;
                if (pd) { R->lo = l.o; R->lm = lm; }
                R->dist = s.dist;
                R->tw = twr;
                R->cost = L == 0 ? 0 : s.dist + d.wL * max(lm - d.Q, 0) + wTe * twr;
            }
        }
        carry = shfl_seg_idx(s, 31);
        if (pd) lcarry = shfl_ld_idx(l, 31);
        have = true;
    }
    // ---- backward scan: suffix after each anchor
    have = false;
    const int nch = (E + 31) >> 5;
    for (int c = nch - 1; c >= 0; --c) {
        const int k = c * 32 + lane;
        const bool valid = k < E;
        const int x = valid ? route_node(d, st, L, k) : 0;
        const int nx = (k + 1 < E) ? route_node(d, st, L, k + 1) : 0;
        const int out = (valid && k + 1 < E) ? dmat(d, x, nx) : 0;
        Seg s = seg_node(d, x, out);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            Seg o = shfl_seg_down(s, off);
            if (lane + off < 32 && k + off < E) s = seg_cat(s, o);
        }
        if (have && valid) s = seg_cat(s, carry);
        Ld l{0, 0, 0};
        if (pd) {
            l = ld_node(d, x);
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const Ld o = shfl_ld_down(l, off);
                if (lane + off < 32 && k + off < E) l = ld_cat(l, o);
            }
            if (have && valid) l = ld_cat(l, lcarry);
        }
        if (valid && k >= 1) {
            const int a = route_anchor(d, r, st, L, k - 1);
            BRec *b = d.brec + TGA_IX(a, d.W + 1);
            b->Lg = tw ? s.L : 0;
            b->twg = tw ? s.TW : 0;
            b->distg = s.dist;
            b->loadg = s.load;
            if (pd) b->lmg = l.m;
        }
        carry = shfl_seg_idx(s, 0);
        if (pd) lcarry = shfl_ld_idx(l, 0);
        have = true;
    }
    __syncwarp();
    // ---- hoisted constants per anchor
    const RouteRec R = d.rrec[TGA_IX(r, d.m)];
    const unsigned mask = d.op_mask;
    const int Q = d.Q;
    for (int k = lane; k <= L; k += 32) {
        const int a = route_anchor(d, r, st, L, k);
        const int x = k == 0 ? 0 : a;
        const BRec b = d.brec[TGA_IX(a, d.W + 1)];
        ERec e;
        PRec pr{};
        e.route = r; e.anchor = a; e.node = x; e.idx = k;
        e.succ = k + 1 <= L ? route_node(d, st, L, k + 1) : 0;
        e.succ2 = k + 2 <= L ? route_node(d, st, L, k + 2) : 0;
        d.brec[TGA_IX(a, d.W + 1)].rlen = L;
        d.brec[TGA_IX(a, d.W + 1)].rcost = R.cost;
        e.d = __ldg(d.demand + x);
        e.e = tw ? __ldg(d.early + x) : 0;
        e.l = tw ? __ldg(d.late + x) : 0;
        e.s = tw ? __ldg(d.service + x) : 0;
        e.tau = b.tau;
        e.Lg = b.Lg;
        const int Fc = b.distf + wTe * b.twf - R.cost;
        const int Gc = b.distg + wTe * b.twg;
        e.K1 = Fc + Gc;
        e.Fc = Fc + ((mask & 8u) ? 0 : kBig);
        e.Gc = Gc;
        e.LQ = R.load - Q;
        e.loadf = b.loadf;
        e.loadgQ = b.loadg - Q;
        e.C2 = kBig; e.ld2 = 0; e.E2 = 0; e.L2 = 0; e.Dm2 = 0;
        e.C3 = kBig; e.ld3 = 0; e.E3 = 0; e.L3 = 0; e.Dm3 = 0;
        if (pd) {
            pr.pk = __ldg(d.pickup + x);
            pr.mx = max(e.d, pr.pk);
            pr.IA = b.lmf + b.loadg - Q; pr.IB = b.lof + b.loadg - Q; pr.IC = b.lof + b.lmg - Q;
            pr.HM = b.lmf - Q; pr.HO = b.lof - Q; pr.TI = b.loadg; pr.TM = b.lmg;
        }
        if (k == 0) {
            e.rem1 = kBig; e.K2 = kBig; e.LQd = 0; e.tauP = 0;
            if (XS) d.xrec[TGA_IX(a, d.W + 1)] = xrec_none();
        } else {
            const int xm = route_node(d, st, L, k - 1);
            const BRec bp = d.brec[TGA_IX(route_anchor(d, r, st, L, k - 1), d.W + 1)];
            const int xn = route_node(d, st, L, k + 1);
            const int cmn = dmat(d, xm, xn);
            if (XS) {
                const bool has1 = k + 1 <= L;
                Seg run{};
                int d1 = 0, g1dist = 0, g1tw = 0, g1L = 0;
                if (has1) {
                    run = seg_cat(seg_node(d, x, dmat(d, x, xn)), seg_node(d, xn, 0));
                    const BRec b1 = d.brec[TGA_IX(xn, d.W + 1)];
                    d1 = __ldg(d.demand + xn);
                    g1dist = b1.distg; g1tw = b1.twg; g1L = b1.Lg;
                }
                d.xrec[TGA_IX(a, d.W + 1)] = make_xrec(wTe, R.cost, R.load, Q, bp.distf, bp.twf, bp.tau, b.distg, b.twg, b.Lg, has1,
                                      g1dist, g1tw, g1L, run, d1, e.e, e.l, e.s, e.d);
            }
            const int twr = tw ? bp.twf + b.twg + max(bp.tau + cmn - b.Lg, 0) : 0;
            // load of the route without x: prefix through x- + suffix after x
            const int lrem = pd ? max(bp.lmf + b.loadg, bp.lof + b.lmg) : R.load - e.d;
            const int c1 = bp.distf + cmn + b.distg + d.wL * max(lrem - Q, 0) + wTe * twr;
            e.rem1 = c1 - R.cost + ((mask & 1u) ? 0 : kBig);
            e.K2 = bp.distf + b.distg + wTe * (bp.twf + b.twg) - R.cost + ((mask & 2u) ? 0 : kBig);
            e.LQd = R.load - e.d - Q;
            e.tauP = bp.tau;
            if (pd) {
                pr.SA = bp.lmf + b.loadg - Q; pr.SB = bp.lof + b.loadg - Q; pr.SC = bp.lof + b.lmg - Q;
            }
            for (int K = 2; K <= 3; ++K) {
                if (k + K - 1 > L || !(mask & (1u << (K + 2)))) continue;
                Seg run = seg_node(d, x, dmat(d, x, route_node(d, st, L, k + 1)));
                Ld rl{0, 0, 0};
                if (pd) rl = ld_node(d, x);
                for (int t = 1; t < K; ++t) {
                    const int y = route_node(d, st, L, k + t);
                    run = seg_cat(run, seg_node(d, y, dmat(d, y, route_node(d, st, L, k + t + 1))));
                    if (pd) rl = ld_cat(rl, ld_node(d, y));
                }
                const int w = route_node(d, st, L, k + K - 1);
                const BRec bw = d.brec[TGA_IX(w, d.W + 1)];
                const int wn = route_node(d, st, L, k + K);
                const int c2 = dmat(d, xm, wn);
                const int twk = tw ? bp.twf + bw.twg + max(bp.tau + c2 - bw.Lg, 0) : 0;
                const int lk = pd ? max(bp.lmf + bw.loadg, bp.lof + bw.lmg) : R.load - run.load;
                const int ck = bp.distf + c2 + bw.distg + d.wL * max(lk - Q, 0) + wTe * twk - R.cost;
                const int CK = ck + run.dist + wTe * (tw ? run.TW : 0);
                if (K == 2) {
                    e.C2 = CK; e.ld2 = run.load;
                    e.E2 = tw ? run.E : 0; e.L2 = tw ? run.L : 0; e.Dm2 = tw ? run.D - run.TW : 0;
                    pr.LO2 = rl.o; pr.LM2 = rl.m;
                } else {
                    e.C3 = CK; e.ld3 = run.load;
                    e.E3 = tw ? run.E : 0; e.L3 = tw ? run.L : 0; e.Dm3 = tw ? run.D - run.TW : 0;
                    pr.LO3 = rl.o; pr.LM3 = rl.m;
                }
            }
        }
        d.erec[TGA_IX(a, d.W + 1)] = e;
        if (pd) d.prec[TGA_IX(a, d.W + 1)] = pr;
    }
}

// Integer headroom: a route built from two current routes plus three moved
// customers must cost below 2^27 (bound from the longest route, heaviest load
// and the largest distance, window and service).  With pickups "load" is
// delivery plus pickup, which bounds every load on board.
__device__ bool range_ok_vals(const Dev &d, int maxL, int maxLoad, int maxc, int maxl, int maxe, int maxs,
                              int maxd) {
    if (maxc >= (1 << 24) || maxl >= (1 << 24) || maxe >= (1 << 24) || maxs >= (1 << 24) || maxd >= (1 << 24))
        return false;
    const long long L2 = 2LL * maxL + 4;
    long long b = L2 * maxc + (long long)d.wL * (2LL * maxLoad + 3LL * maxd);
    if (d.has_tw) b += (long long)d.wT * L2 * ((long long)maxl + maxs + maxc);
    return b < kRouteCostLim;
}

__device__ bool range_ok(const Dev &d, const Control *C) {
    return range_ok_vals(d, C->maxL, C->maxLoad, C->maxc, C->maxl, C->maxe, C->maxs, C->maxd);
}

// ---------------------------------------------------------------------------
// build

// Symmetry / diagonal / sign check of the distance matrix, tile by tile:
// block (32 x 8 threads) loads tile (I, J) and tile (J, I) with coalesced row
// reads into shared memory and compares one against the transpose of the other.
__device__ void check_instance_tiles(const Dev &d, int part, int nparts) {
    Control *C = d.ctl;
    __shared__ int A[32][33], B[32][33];
    const int n1 = d.n + 1, nt = (n1 + 31) / 32;
    const long long ntiles = (long long)nt * nt;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    int mx = 0;
    bool bad = false;
    const int nwarps = blockDim.x >> 5;
    for (long long t = part; t < ntiles; t += nparts) {
        const int I = (int)(t / nt), J = (int)(t - (long long)I * nt);
        for (int rr = ty; rr < 32; rr += nwarps) {
            const int i = I * 32 + rr, j = J * 32 + tx;
            A[rr][tx] = (i < n1 && j < n1) ? d.dist[(size_t)i * n1 + j] : 0;
            const int i2 = J * 32 + rr, j2 = I * 32 + tx;
            B[rr][tx] = (i2 < n1 && j2 < n1) ? d.dist[(size_t)i2 * n1 + j2] : 0;
        }
        __syncthreads();
        for (int rr = ty; rr < 32; rr += nwarps) {
            const int i = I * 32 + rr, j = J * 32 + tx;
            if (i < n1 && j < n1) {
                const int v = A[rr][tx];
                if (v < 0 || (i == j && v != 0) || v != B[tx][rr]) bad = true;
                mx = max(mx, v);
            }
        }
        __syncthreads();
    }
    int md = 0, ml = 0, ms = 0, me = 0;
    for (long long i = part * (long long)blockDim.x + threadIdx.x; i < n1;
         i += (long long)nparts * blockDim.x) {
        const int dm = d.demand[i];
        if (dm < 0 || (i == 0 && dm != 0)) bad = true;
        md = max(md, dm);
        if (d.has_pd) {                        // range bound: delivery plus pickup
            const int pk = d.pickup[i];
            if (pk < 0 || (i == 0 && pk != 0)) bad = true;
            md = max(md, dm + pk);
        }
        if (d.has_tw) {
            const int e = d.early[i], l = d.late[i], sv = d.service[i];
            if (e < 0 || l < 0 || sv < 0 || (i == 0 && sv != 0)) bad = true;
            ml = max(ml, l); ms = max(ms, sv); me = max(me, e);
        }
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    md = __reduce_max_sync(0xffffffffu, md);
    ml = __reduce_max_sync(0xffffffffu, ml);
    ms = __reduce_max_sync(0xffffffffu, ms);
    me = __reduce_max_sync(0xffffffffu, me);
    const bool anybad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&C->maxc, mx); atomicMax(&C->maxd, md); atomicMax(&C->maxl, ml);
        atomicMax(&C->maxs, ms); atomicMax(&C->maxe, me);
        if (anybad) set_status(C, TGA_ERR_INVALID);
    }
}

__device__ void build_positions_route(const Dev &d, int r) {
    Control *C = d.ctl;
    if (r == 0) {
        if (d.route_start[TGA_IX(0, d.m + 1)] != 0 || d.route_start[TGA_IX(d.m, d.m + 1)] != d.n) set_status(C, TGA_ERR_INVALID);
        d.seq[TGA_IX(d.n + d.m, d.Wp)] = d.W;   // sentinel (end depot of the last route)
    }
    if (r >= d.m) return;
    const int a = d.route_start[TGA_IX(r, d.m + 1)], b = d.route_start[TGA_IX(r + 1, d.m + 1)];
    if (a < 0 || b < a || b > d.n) { set_status(C, TGA_ERR_INVALID); return; }
    const int p = a + r;
    d.seq[TGA_IX(p, d.Wp)] = d.n + 1 + r;
    d.pos_of[TGA_IX(d.n + 1 + r, d.W + 1)] = p;
    d.rrec[TGA_IX(r, d.m)].start = p;
    d.rrec[TGA_IX(r, d.m)].len = b - a;
    for (int t = a; t < b; ++t) {
        const int x = d.tour[TGA_IX(t, d.n)];
        if (x < 1 || x > d.n) { set_status(C, TGA_ERR_INVALID); continue; }
        d.seq[TGA_IX(t + r + 1, d.Wp)] = x;
        d.pos_of[TGA_IX(x, d.W + 1)] = t + r + 1;
        atomicAdd(&d.seen[TGA_IX(x, d.n + 1)], 1);
    }
}

__device__ __forceinline__ void check_perm_one(const Dev &d, int x) {
    if (x >= 1 && x <= d.n && d.seen[TGA_IX(x, d.n + 1)] != 1) set_status(d.ctl, TGA_ERR_INVALID);
}


__device__ void finish_block(const Dev &d) {
    Control *C = d.ctl;
    __shared__ long long s_cost[32], s_l2[32], s_l1[32], s_lm2[32], s_q1[32], s_q2[32];
    __shared__ int s_maxL[32], s_maxLoad[32];
    long long cost = 0, l2 = 0, l1 = 0, lm2 = 0, q1 = 0, q2 = 0;
    int maxL = 0, maxLoad = 0;
    if (C->status == 0) {
        for (int r = threadIdx.x; r < d.m; r += blockDim.x) {
            const RouteRec R = d.rrec[TGA_IX(r, d.m)];
            cost += R.cost;
            l2 += (long long)R.len * R.len;
            l1 += max(R.len - 1, 0);
            lm2 += max(R.len - 2, 0);
            q1 += (long long)max(R.len - 1, 0) * max(R.len - 1, 0);
            q2 += (long long)max(R.len - 2, 0) * max(R.len - 2, 0);
            maxL = max(maxL, R.len);
            maxLoad = max(maxLoad, d.has_pd ? R.load + R.lo : R.load);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        cost += __shfl_xor_sync(0xffffffffu, cost, off);
        l2 += __shfl_xor_sync(0xffffffffu, l2, off);
        l1 += __shfl_xor_sync(0xffffffffu, l1, off);
        lm2 += __shfl_xor_sync(0xffffffffu, lm2, off);
        q1 += __shfl_xor_sync(0xffffffffu, q1, off);
        q2 += __shfl_xor_sync(0xffffffffu, q2, off);
        maxL = max(maxL, __shfl_xor_sync(0xffffffffu, maxL, off));
        maxLoad = max(maxLoad, __shfl_xor_sync(0xffffffffu, maxLoad, off));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        s_cost[warp] = cost; s_l2[warp] = l2; s_l1[warp] = l1; s_lm2[warp] = lm2;
        s_q1[warp] = q1; s_q2[warp] = q2;
        s_maxL[warp] = maxL; s_maxLoad[warp] = maxLoad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
            cost += s_cost[w]; l2 += s_l2[w]; l1 += s_l1[w]; lm2 += s_lm2[w];
            q1 += s_q1[w]; q2 += s_q2[w];
            maxL = max(maxL, s_maxL[w]); maxLoad = max(maxLoad, s_maxLoad[w]);
        }
        C->cost = cost; C->initial_cost = cost;
        C->sumL2 = l2; C->sumLm1 = l1; C->sumLm2 = lm2;
        C->sumLm1sq = q1; C->sumLm2sq = q2;
        for (int op = 0; op < 6; ++op) C->gcount[op] = 0;
        C->maxL = maxL; C->maxLoad = maxLoad;
        C->steps = 0; C->evals = 0; C->cand_total = 0;
        for (int op = 0; op < 8; ++op) C->cand_op[op] = 0;
        C->done = 0; C->local_opt = 0;
        C->plan_ready = 0; C->plan_done = 0;
        C->best_key = kNoKey;
        C->step_limit = 0x7fffffffffffffffLL;
        C->cand_per_eval = candidate_count(d.n, d.m, d.op_mask, l2, l1, lm2);
        if (C->status == 0 && !range_ok(d, C)) set_status(C, TGA_ERR_RANGE);
        if (C->status != 0) C->done = 1;
        C->built = 1;
        // dummy record (sentinel position and every position past the end)
        ERec e{};
        e.route = -1; e.anchor = d.W;
        e.rem1 = kBig; e.K1 = kBig; e.K2 = kBig; e.Fc = kBig; e.C2 = kBig; e.C3 = kBig;
        d.erec[TGA_IX(d.W, d.W + 1)] = e;
        BRec b{};
        b.route = -1;
        d.brec[TGA_IX(d.W, d.W + 1)] = b;
        if (d.has_pd) d.prec[TGA_IX(d.W, d.W + 1)] = PRec{};
        if (d.op_mask & kExtOps) d.xrec[TGA_IX(d.W, d.W + 1)] = xrec_none();
    }
}

// pcol[x][q + kColOff] = dist[x][node at position q]; columns outside the
// position range hold the depot distance (read only by masked candidates).
__device__ void pcol_init_range(const Dev &d, long long t0, long long stride) {
    const long long tot = (long long)(d.n + 1) * d.ldp;
    for (long long t = t0; t < tot; t += stride) {
        const int x = (int)(t / d.ldp), c = (int)(t - (long long)x * d.ldp);
        const int q = c - kColOff;
        const int node = (q >= 0 && q < d.Wp) ? node_of(d.seq[TGA_IX(q, d.Wp)], d.n) : 0;
        d.pcol[TGA_IX(t, (long long)(d.n + 1) * d.ldp)] = dmat(d, x, node);
    }
}

// ---------------------------------------------------------------------------
// inter-route evaluation

#define TGA_TRY(dl, ix)                                                    \
    do {                                                                   \
        const int _d = (dl);                                               \
        const unsigned _i = (ix);                                          \
        if (_d < best || (_d == best && _i < bidx)) { best = _d; bidx = _i; } \
    } while (0)

// Tile number bid of the inter-route pair triangle, in the order of the
// host's tile list: row tiles I = 0.. (TR rows each), and in row tile I the
// column tiles J = floor(I/g) .. nct-1 (g = TC/TR, an integer: the first
// column tile holding a pair p < q).  The number of tiles before row tile I
// has a closed form, so I is found by binary search with no memory access.
__device__ __forceinline__ int2 tile_of(int bid, int Wp, int TR, int TC) {
    const int Wa = Wp - 1;
    const int nrt = (Wa + TR - 1) / TR, nct = (Wa + TC - 1) / TC, g = TC / TR;
    auto before = [&](int I) -> long long {
        const long long q = I / g, r = I - q * g;
        return (long long)I * nct - ((long long)g * q * (q - 1) / 2 + r * q);
    };
    int lo = 0, hi = nrt - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (before(mid) <= bid) lo = mid;
        else hi = mid - 1;
    }
    return make_int2(lo, lo / g + (int)(bid - before(lo)));
}

// Asynchronous global -> shared copies of 16 bytes (cp.async, L2 only: the
// copies read what other SMs wrote before the last grid-wide hand-off).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The column side of an inter-route tile: the anchor av at position q and
// its hoisted constants (ERec groups; PRec with pickups), held in registers
// while a warp walks the rows.
struct InterCol {
    int q, av;
    int4 v0, v1, v2, v3, v4, v5, v6;
    int4 w0, w1, w2, w3;
};

template <bool TW, bool OR, bool PD>
__device__ __forceinline__ void inter_col_fill(const Dev &d, int q, int av, InterCol &c) {
    c.q = q;
    c.av = av;
    const int4 *vr = reinterpret_cast<const int4 *>(d.erec + TGA_IX(c.av, d.W + 1));
    c.v0 = TGA_LDG(vr + 0); c.v1 = TGA_LDG(vr + 1); c.v2 = TGA_LDG(vr + 2);
    c.v3 = make_int4(0, 0, 0, 0); c.v4 = c.v3; c.v5 = c.v3; c.v6 = c.v3;
    if (OR) c.v3 = TGA_LDG(vr + 3);
    if (TW) { c.v4 = TGA_LDG(vr + 4); c.v5 = TGA_LDG(vr + 5); }
    if (TW && OR) c.v6 = TGA_LDG(vr + 6);
    c.w0 = make_int4(0, 0, 0, 0); c.w1 = c.w0; c.w2 = c.w0; c.w3 = c.w0;
    if (PD) {
        const int4 *pr = reinterpret_cast<const int4 *>(d.prec + TGA_IX(c.av, d.W + 1));
        c.w0 = TGA_LDG(pr + 0); c.w1 = TGA_LDG(pr + 1); c.w2 = TGA_LDG(pr + 2);
        if (OR) c.w3 = TGA_LDG(pr + 3);
    }
}

template <bool TW, bool OR, bool PD>
__device__ __forceinline__ void inter_col_load(const Dev &d, int q, InterCol &c) {
    inter_col_fill<TW, OR, PD>(d, q, (q < d.Wp) ? d.seq[TGA_IX(q, d.Wp)] : d.W, c);
}

// Rows i0..i1-1 of a staged tile against one column: row i is the anchor at
// position p0 + i with its records at sR[i*NG ..] (ERec groups, then PRec
// with pickups); col points at the column's distance in the tile's row
// "p0 - 1" (row stride LDT), so row i's stencil sits at col[(i+1)*LDT + ...].
// Every candidate of every pair with p < q in different routes is folded
// into (best, bidx).  UNR: row-loop unrolling (lets the compiler issue the
// next rows' shared loads early; the strip kernel gains from it, the
// one-wave persistent descent does not).
template <bool TW, bool OR, bool PD = false, int UNR = 1, bool GATE = false>
__device__ __forceinline__ void inter_rows(const Dev &d, const InterCol &c, const int *col, const int4 *sR, int LDT,
                                           int p0, int i0, int i1, int &best, unsigned &bidx) {
    constexpr int NG = PD ? 12 : 8;                           // int4 records per row
    const int q = c.q, av = c.av;
    const int4 v0 = c.v0, v1 = c.v1, v2 = c.v2, v3 = c.v3, v4 = c.v4, v5 = c.v5, v6 = c.v6;
    const int4 w0 = c.w0, w1 = c.w1, w2 = c.w2, w3 = c.w3;
    // column fields
    const int Vroute = v0.x, Vd = v0.y, Vrem1 = v0.z, VK1 = v0.w;
    const int VLQ = v1.x, VK2 = v1.y, VLQd = v1.z, VFc = v1.w;
    const int VGc = v2.x, Vloadf = v2.y, VloadgQ = v2.z;
    const int VC2 = v3.x, Vld2 = v3.y, VC3 = v3.z, Vld3 = v3.w;
    const int Ve = v4.x, Vl = v4.y, Vs = v4.z, Vtau = v4.w;
    const int VLg = v5.x, VtauP = v5.y, VE2 = v5.z, VL2 = v5.w;
    const int VDm2 = v6.x, VE3 = v6.y, VL3 = v6.z, VDm3 = v6.w;
    (void)w3;
    const int wL = d.wL, wT = d.wT;
    const unsigned W = (unsigned)d.W, W2 = W * W;
    const int *c0 = col + i0 * LDT;                           // window at row i0
    int tm10 = c0[0];
    int t0m1 = c0[LDT - 1], t00 = c0[LDT], t01 = c0[LDT + 1];
    int t10 = c0[2 * LDT], t11 = c0[2 * LDT + 1], t12 = c0[2 * LDT + 2];
    int t21 = c0[3 * LDT + 1];
    int wbest = __reduce_min_sync(0xffffffffu, best);
    // GATE: skip the operators the mask disables (their deltas stay kBig,
    // above every valid delta); without it every operator of the variant is
    // on and the code is the ungated one
    const unsigned mk = d.op_mask;
    const bool onR = !GATE || (mk & 1u), onS = !GATE || (mk & 2u), onX = !GATE || (mk & 8u);
    const bool onO2 = !GATE || (mk & 16u), onO3 = !GATE || (mk & 32u);

#pragma unroll UNR
    for (int i = i0; i < i1; ++i) {
        const int p = p0 + i;
        const int4 u0 = sR[i * NG + 0], u1 = sR[i * NG + 1], u2 = sR[i * NG + 2];
        const int Uroute = u0.x, Ud = u0.y, Urem1 = u0.z, UK1 = u0.w;
        const int ULQ = u1.x, UK2 = u1.y, ULQd = u1.z, UFc = u1.w;
        const int UGc = u2.x, Uloadf = u2.y, UloadgQ = u2.z;
        // distances of the stencil (symmetric matrix):
        //   c(u,v)=t00 c(u,v+)=t01 c(u+,v)=t10 c(u+,v+)=t11 c(u++,v+)=t21
        //   c(u+,v++)=t12 c(u-,v)=tm10 c(u,v-)=t0m1
        // relocate u -> after v, relocate v -> after u
        // (with pickups the load terms follow below)
        int dR1 = kBig, dR2 = kBig, dS = kBig, dX = kBig;
        if (onR) {
            dR1 = Urem1 + VK1 + t00 + t01 + (PD ? 0 : wL * max(VLQ + Ud, 0));
            dR2 = Vrem1 + UK1 + t00 + t10 + (PD ? 0 : wL * max(ULQ + Vd, 0));
        }
        // swap u <-> v
        if (onS)
            dS = UK2 + VK2 + tm10 + t10 + t0m1 + t01 + (PD ? 0 : wL * (max(ULQd + Vd, 0) + max(VLQd + Ud, 0)));
        // 2-opt*: head(u)+tail after v, head(v)+tail after u
        if (onX)
            dX = UFc + VGc + VFc + UGc + t01 + t10 +
                 (PD ? 0 : wL * (max(Uloadf + VloadgQ, 0) + max(Vloadf + UloadgQ, 0)));
        int dO2a = kBig, dO2b = kBig, dO3a = kBig, dO3b = kBig;
        int4 u3 = make_int4(0, 0, 0, 0);
        if (OR) {
            u3 = sR[i * NG + 3];
            const int UC2 = u3.x, Uld2 = u3.y, UC3 = u3.z, Uld3 = u3.w;
            if (onO2) {
                dO2a = UC2 + VK1 + t00 + t11 + (PD ? 0 : wL * max(VLQ + Uld2, 0));
                dO2b = VC2 + UK1 + t00 + t11 + (PD ? 0 : wL * max(ULQ + Vld2, 0));
            }
            if (onO3) {
                dO3a = UC3 + VK1 + t00 + t21 + (PD ? 0 : wL * max(VLQ + Uld3, 0));
                dO3b = VC3 + UK1 + t00 + t12 + (PD ? 0 : wL * max(ULQ + Vld3, 0));
            }
        }
        if (PD) {
            // largest loads of the new routes (Section 4.3.2) from the PRec
            // constants: insertion after an anchor, a customer in place of
            // another, and the 2-opt* recombinations
            const int4 x0 = sR[i * NG + 8], x1 = sR[i * NG + 9], x2 = sR[i * NG + 10];
            const int UIA = x0.x, UIB = x0.y, UIC = x0.z, Upk = x0.w;
            const int USA = x1.x, USB = x1.y, USC = x1.z, Umx = x1.w;
            const int UHM = x2.x, UHO = x2.y, UTI = x2.z, UTM = x2.w;
            const int VIA = w0.x, VIB = w0.y, VIC = w0.z, Vpk = w0.w;
            const int VSA = w1.x, VSB = w1.y, VSC = w1.z, Vmx = w1.w;
            const int VHM = w2.x, VHO = w2.y, VTI = w2.z, VTM = w2.w;
            if (onR) {
                dR1 += wL * max(max(max(VIA + Ud, VIB + Umx), VIC + Upk), 0);
                dR2 += wL * max(max(max(UIA + Vd, UIB + Vmx), UIC + Vpk), 0);
            }
            if (onS)
                dS += wL * (max(max(max(USA + Vd, USB + Vmx), USC + Vpk), 0) +
                            max(max(max(VSA + Ud, VSB + Umx), VSC + Upk), 0));
            if (onX) dX += wL * (max(max(UHM + VTI, UHO + VTM), 0) + max(max(VHM + UTI, VHO + UTM), 0));
            if (OR) {
                const int4 x3 = sR[i * NG + 11];
                const int ULO2 = x3.x, ULM2 = x3.y, ULO3 = x3.z, ULM3 = x3.w;
                const int VLO2 = w3.x, VLM2 = w3.y, VLO3 = w3.z, VLM3 = w3.w;
                const int Uld2 = u3.y, Uld3 = u3.w;
                if (onO2) {
                    dO2a += wL * max(max(max(VIA + Uld2, VIB + ULM2), VIC + ULO2), 0);
                    dO2b += wL * max(max(max(UIA + Vld2, UIB + VLM2), UIC + VLO2), 0);
                }
                if (onO3) {
                    dO3a += wL * max(max(max(VIA + Uld3, VIB + ULM3), VIC + ULO3), 0);
                    dO3b += wL * max(max(max(UIA + Vld3, UIB + VLM3), UIC + VLO3), 0);
                }
            }
        }
        const bool skip = (Uroute == Vroute) | (p >= q);
        // Every time-window term below adds a non-negative warp penalty, so
        // the deltas without them bound the pair's deltas from below.  When
        // no lane's bound can tie or beat the warp's best so far, no
        // candidate of this row can hold the argmin: the terms are skipped
        // for the whole warp, and the minimum test further down then fails
        // for every lane, exactly as it would with the terms added.
        int lb = min(min(dR1, dR2), min(dS, dX));
        if (OR) lb = min(lb, min(min(dO2a, dO2b), min(dO3a, dO3b)));
        if (TW && __any_sync(0xffffffffu, !skip && lb <= wbest)) {
            const int4 u4 = sR[i * NG + 4], u5 = sR[i * NG + 5];
            const int Ue = u4.x, Ul = u4.y, Us = u4.z, Utau = u4.w;
            const int ULg = u5.x, UtauP = u5.y;
            if (onR) {   // u inserted between v and v+
                const int a1 = Vtau + t00, w1 = max(a1 - Ul, 0);
                const int a2 = max(a1, Ue) - w1 + Us + t01, w2 = max(a2 - VLg, 0);
                dR1 += wT * (w1 + w2);
            }
            if (onR) {   // v inserted between u and u+
                const int a1 = Utau + t00, w1 = max(a1 - Vl, 0);
                const int a2 = max(a1, Ve) - w1 + Vs + t10, w2 = max(a2 - ULg, 0);
                dR2 += wT * (w1 + w2);
            }
            if (onS) {   // v between u- and u+, u between v- and v+
                const int a1 = UtauP + tm10, w1 = max(a1 - Vl, 0);
                const int a2 = max(a1, Ve) - w1 + Vs + t10, w2 = max(a2 - ULg, 0);
                const int b1 = VtauP + t0m1, x1 = max(b1 - Ul, 0);
                const int b2 = max(b1, Ue) - x1 + Us + t01, x2 = max(b2 - VLg, 0);
                dS += wT * (w1 + w2 + x1 + x2);
            }
            if (onX) dX += wT * (max(Utau + t01 - VLg, 0) + max(Vtau + t10 - ULg, 0));
            if (OR) {
                const int UE2 = u5.z, UL2 = u5.w;
                const int4 u6 = sR[i * NG + 6];
                const int UDm2 = u6.x, UE3 = u6.y, UL3 = u6.z, UDm3 = u6.w;
                if (onO2) {
                    const int a1 = Vtau + t00, w1 = max(a1 - UL2, 0);
                    const int a2 = max(a1, UE2) - w1 + UDm2 + t11, w2 = max(a2 - VLg, 0);
                    dO2a += wT * (w1 + w2);
                }
                if (onO2) {
                    const int a1 = Utau + t00, w1 = max(a1 - VL2, 0);
                    const int a2 = max(a1, VE2) - w1 + VDm2 + t11, w2 = max(a2 - ULg, 0);
                    dO2b += wT * (w1 + w2);
                }
                if (onO3) {
                    const int a1 = Vtau + t00, w1 = max(a1 - UL3, 0);
                    const int a2 = max(a1, UE3) - w1 + UDm3 + t21, w2 = max(a2 - VLg, 0);
                    dO3a += wT * (w1 + w2);
                }
                if (onO3) {
                    const int a1 = Utau + t00, w1 = max(a1 - VL3, 0);
                    const int a2 = max(a1, VE3) - w1 + VDm3 + t12, w2 = max(a2 - ULg, 0);
                    dO3b += wT * (w1 + w2);
                }
            }
        }
        int m = min(min(dR1, dR2), min(dS, dX));
        if (OR) m = min(m, min(min(dO2a, dO2b), min(dO3a, dO3b)));
        // Only a pair that can tie or beat the warp's best so far can hold the
        // final argmin (every lane's best bounds the global minimum from
        // above), so the packed keys are formed only then; filtering on the
        // warp minimum rather than the lane's own keeps the whole warp off
        // this path on almost every row.
        if (!skip && m <= wbest) {
            // the pair's best candidate: the first, in move-index order, whose
            // delta is the minimum m (op rank first; within relocate and the
            // or-opts the move of the lower anchor id first)
            const unsigned au = (unsigned)u2.w, avu = (unsigned)av;
            const bool uf = au < avu;
            const unsigned lo = uf ? au : avu, hi = uf ? avu : au;
            unsigned op = 5, A = hi, B = lo;
            if ((uf ? dR1 : dR2) == m) { op = 0; A = lo; B = hi; }
            else if ((uf ? dR2 : dR1) == m) { op = 0; A = hi; B = lo; }
            else if (dS == m) { op = 1; A = lo; B = hi; }
            else if (dX == m) { op = 3; A = Uroute < Vroute ? au : avu; B = Uroute < Vroute ? avu : au; }
            else if (OR && (uf ? dO2a : dO2b) == m) { op = 4; A = lo; B = hi; }
            else if (OR && (uf ? dO2b : dO2a) == m) { op = 4; A = hi; B = lo; }
            else if (OR && (uf ? dO3a : dO3b) == m) { op = 5; A = lo; B = hi; }
            TGA_TRY(m, op * W2 + A * W + B);
        }
        wbest = __reduce_min_sync(0xffffffffu, best);
        // slide the stencil window one row down
        tm10 = t00;
        t0m1 = col[(i + 2) * LDT - 1];
        t00 = t10;
        t01 = t11;
        t10 = col[(i + 3) * LDT];
        t11 = t21;
        t12 = col[(i + 3) * LDT + 2];
        t21 = col[(i + 4) * LDT + 1];
    }
}

// One tile of the inter-route pair triangle: rows p0..p0+TR-1, columns
// q0..q0+32*NWc-1 with NWc = warps / RS.  Warp w owns the 32 columns of slice
// w % NWc and the rows of group w / NWc (TR/RS rows each).  Every thread folds
// its column's candidates into (best, bidx); smem must hold
// inter_smem_bytes(TR, NWc, PD).  PD: pickups (requires TW); every load
// excess is that of the new route's largest load (PRec constants).
template <bool TW, bool OR, bool PD = false, bool GATE = false>
__device__ void inter_tile(const Dev &d, int p0, int q0, int TR, int RS, int *smem, int &best, unsigned &bidx) {
    constexpr int NG = PD ? 12 : 8;                           // int4 records per row
    const int NW = blockDim.x >> 5, NWc = NW / RS, TC = NWc * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cw = warp % NWc, rg = warp / NWc, rows_per = TR / RS;
    const int i0 = rg * rows_per, i1 = i0 + rows_per;
    const int LDT = TC + 8;
    int *sT = smem;                                           // (TR+4) x LDT distances
    int4 *sR = reinterpret_cast<int4 *>(smem + (TR + 4) * LDT);   // TR row records (ERec, then PRec)
    __shared__ int s_rnode[68];                               // nodes of positions p0-1 .. p0+TR+2 (TR <= 64)
    __shared__ int s_ranc[64];                                // anchors of positions p0 .. p0+TR-1
    // first loads: the anchors of the rows and of this thread's column
    const int q = q0 + cw * 32 + lane;
    const int av = (q < d.Wp) ? d.seq[TGA_IX(q, d.Wp)] : d.W;
    __syncthreads();                                          // previous user of smem is done
    for (int t = threadIdx.x; t < TR + 4; t += blockDim.x) {
        const int p = p0 - 1 + t;
        const bool in = p >= 0 && p < d.Wp;
        const int a = in ? d.seq[TGA_IX(p, d.Wp)] : d.W;
        s_rnode[t] = in ? node_of(a, d.n) : 0;
        if (t >= 1 && t <= TR) s_ranc[t - 1] = a;
    }
    __syncthreads();
    // second loads, all issued before any is waited for: the extraction rows
    // p0-1 .. p0+TR+2 over positions q0-4 .. q0+TC+3 and the row records
    // (asynchronous copies), and the column's records (registers)
    const int C4 = LDT >> 2;
    for (int i = threadIdx.x; i < (TR + 4) * C4; i += blockDim.x) {
        const int rr = i / C4, c4 = i - rr * C4;
        cp_async16(sT + rr * LDT + 4 * c4,
                   d.pcol + (size_t)TGA_IX(s_rnode[rr], d.n + 1) * d.ldp + TGA_IX(q0 + 4 * c4, d.ldp - 3));
    }
    for (int i = threadIdx.x; i < TR * NG; i += blockDim.x) {
        const int row = i / NG, g = i - row * NG;
        const int a = s_ranc[row];
        cp_async16(sR + i, g < 8 ? reinterpret_cast<const int4 *>(d.erec + TGA_IX(a, d.W + 1)) + g
                                 : reinterpret_cast<const int4 *>(d.prec + TGA_IX(a, d.W + 1)) + (g - 8));
    }
    cp_async_commit();
    InterCol c;
    inter_col_fill<TW, OR, PD>(d, q, av, c);
    cp_async_wait<0>();
    __syncthreads();
    inter_rows<TW, OR, PD, 1, GATE>(d, c, sT + cw * 32 + lane + 4, sR, LDT, p0, i0, i1, best, bidx);
}

// Anchor at position p for row staging (positions outside the sequence read
// the dummy record W, whose node is the depot).
__device__ __forceinline__ int strip_anchor(const Dev &d, int p) { return (p >= 0 && p < d.Wp) ? d.seq[TGA_IX(p, d.Wp)] : d.W; }

// Issue the copies of one tile: TR+4 distance rows (the nodes of positions
// p0-1 .. p0+TR+2, storage columns q0 .. q0+TC+7, i.e. positions
// q0-4 .. q0+TC+3) and the TR row records (ERec, then PRec with pickups).
template <bool PD>
__device__ __forceinline__ void strip_stage(const Dev &d, int *buf, int TR, int q0, const int *s_anc) {
    constexpr int NG = PD ? 12 : 8;
    const int NW = blockDim.x >> 5, TC = NW * 32, LDT = TC + 8, C4 = LDT >> 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int4 *sR = reinterpret_cast<int4 *>(buf + (TR + 4) * LDT);
    for (int r = warp; r < TR + 4; r += NW) {
        const int node = node_of(s_anc[r], d.n);
        const int4 *src =
            reinterpret_cast<const int4 *>(d.pcol + (size_t)TGA_IX(node, d.n + 1) * d.ldp + TGA_IX(q0, d.ldp - LDT + 1));
        int4 *dst = reinterpret_cast<int4 *>(buf + r * LDT);
        for (int c = lane; c < C4; c += 32) cp_async16(dst + c, src + c);
    }
    for (int i = threadIdx.x; i < TR * NG; i += blockDim.x) {
        const int row = i / NG, g = i - row * NG;
        const int a = s_anc[row + 1];
        const int4 *src = g < 8 ? reinterpret_cast<const int4 *>(d.erec + TGA_IX(a, d.W + 1)) + g
                                : reinterpret_cast<const int4 *>(d.prec + TGA_IX(a, d.W + 1)) + (g - 8);
        cp_async16(sR + i, src);
    }
}

// Walk the tiles t0 .. t1-1 of the strip-major order (TR rows x TC =
// 32 * warps columns each): the anchors of each tile, its copies into one of
// two buffers while the other is computed, the strip's column anchors in
// registers, and the row loop of inter_rows.  smem: strip_smem_bytes(TR,
// warps, PD); every thread of the block calls.  Used by the per-step kernel
// (k_eval_strip) and by the persistent descent's strip mode.
template <bool TW, bool OR, bool PD = false, bool GATE = false, int UNR = TW ? 1 : 4>
__device__ void strip_walk(const Dev &d, int TR, long long T, long long t0, long long t1, int *smem, int &best,
                           unsigned &bidx) {
    constexpr int NG = PD ? 12 : 8;
    const int NW = blockDim.x >> 5, TC = NW * 32, LDT = TC + 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int Wa = d.Wp - 1;
    const int nrt = (Wa + TR - 1) / TR, nct = (Wa + TC - 1) / TC, g = TC / TR;
    const int buf_ints = (TR + 4) * LDT + TR * NG * 4;
    int *s_anc = smem + 2 * buf_ints;                    // two (TR+4)-entry anchor lists (positions p0-1 ..)
    (void)T;
    __syncthreads();                                     // the previous user of smem is done
    if (t0 < t1) {
        // strip and row tile of t0: the last strip that starts at or before t0
        int lo = 0, hi = nct - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (strip_before(mid, nrt, g) <= t0) lo = mid;
            else hi = mid - 1;
        }
        int J = lo, I = (int)(t0 - strip_before(lo, nrt, g));
        auto next = [&](int &j, int &i) {
            if (++i >= min((j + 1) * g, nrt)) { ++j; i = 0; }
        };
        // prologue: anchors of tile t0, its copies, and the anchors of t0 + 1
        if (tid < TR + 4) s_anc[tid] = strip_anchor(d, I * TR - 1 + tid);
        int Jn = J, In = I;
        next(Jn, In);
        int a_next = (t0 + 1 < t1 && tid < TR + 4) ? strip_anchor(d, In * TR - 1 + tid) : 0;
        __syncthreads();
        strip_stage<PD>(d, smem, TR, J * TC, s_anc);
        cp_async_commit();
        InterCol c;
        int Jc = -1;
        for (long long k = t0; k < t1; ++k) {
            const int b = (int)((k - t0) & 1);
            int *cur = smem + b * buf_ints;
            const bool more = k + 1 < t1;
            if (more) {
                int *nanc = s_anc + (b ^ 1) * (TR + 4);
                if (tid < TR + 4) nanc[tid] = a_next;
                __syncthreads();                         // anchors written; the other buffer is free
                strip_stage<PD>(d, smem + (b ^ 1) * buf_ints, TR, Jn * TC, nanc);
                cp_async_commit();
                int Jnn = Jn, Inn = In;
                next(Jnn, Inn);
                if (k + 2 < t1 && tid < TR + 4) a_next = strip_anchor(d, Inn * TR - 1 + tid);
                cp_async_wait<1>();                      // this tile's copies are done
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();                             // ... for every thread of the block
            if (J != Jc) {                               // a new strip: its column anchors
                inter_col_load<TW, OR, PD>(d, J * TC + warp * 32 + lane, c);
                Jc = J;
            }
            inter_rows<TW, OR, PD, UNR, GATE>(d, c, cur + warp * 32 + lane + 4,
                                   reinterpret_cast<const int4 *>(cur + (TR + 4) * LDT), LDT, I * TR, 0, TR,
                                   best, bidx);
            J = Jn; I = In;
            next(Jn, In);
        }
    }
}

// ---------------------------------------------------------------------------
// inter-route evaluation, edge-based extraction (Section 5.3.1): the
// candidates of one pair of a customer u and an anchor v of another route --
// v a customer of u's mask row (a directed mask edge u -> v) or the start
// depot of another route -- with the expressions of inter_tile.  The caller
// supplies u's ERec groups g0..g6, v's groups g0, g1, g2, g4, g5 and the
// stencil distances
//   t00 = c(u, v)   t01 = c(u, v+)   t10 = c(u+, v)   t11 = c(u+, v+)
//   t21 = c(u++, v+)   tm10 = c(u-, v)   t0m1 = c(u, v-)
// (x+ / x- the nodes after / before x in the giant sequence, a depot being
// node 0; tm10 and t0m1 are read only for a customer v).  Kept per pair: u
// and its runs of 2 and 3 moved after v; swap and 2-opt* once per unordered
// customer pair (pair_once); 2-opt* of u with a start depot.  Intra-route
// pairs are left to the route kernels.  Returns a bit mask of the operator
// ranks evaluated (one candidate each).
struct EdgeStencil {
    int t00, t01, t10, t11, t21, tm10, t0m1;
};

template <bool TW, bool OR>
__device__ __forceinline__ unsigned edge_pair(const Dev &d, int u, int v, bool vcust, bool pair_once,
                                              const int4 &u0, const int4 &u1, const int4 &u2, const int4 &u3,
                                              const int4 &u4, const int4 &u5, const int4 &u6, const int4 &v0,
                                              const int4 &v1, const int4 &v2, const int4 &v4, const int4 &v5,
                                              const EdgeStencil &t, int &best, unsigned &bidx) {
    const unsigned mask = d.op_mask;
    const int Uroute = u0.x, Vroute = v0.x;
    unsigned evaluated = 0;
    const int t00 = t.t00, t01 = t.t01, t10 = t.t10, t11 = t.t11, t21 = t.t21, tm10 = t.tm10, t0m1 = t.t0m1;
    const int wL = d.wL, wT = d.wT;
    const unsigned W = (unsigned)d.W, W2 = W * W;
    const int Ud = u0.y, Urem1 = u0.z, UK2 = u1.y, ULQd = u1.z, UFc = u1.w;
    const int UGc = u2.x, Uloadf = u2.y, UloadgQ = u2.z;
    const int Vd = v0.y, VK1 = v0.w, VLQ = v1.x, VK2 = v1.y, VLQd = v1.z, VFc = v1.w;
    const int VGc = v2.x, Vloadf = v2.y, VloadgQ = v2.z;
    const int Ue = u4.x, Ul = u4.y, Us = u4.z, Utau = u4.w, ULg = u5.x, UtauP = u5.y;
    const int Ve = v4.x, Vl = v4.y, Vs = v4.z, Vtau = v4.w, VLg = v5.x, VtauP = v5.y;
    const unsigned au = (unsigned)u, av = (unsigned)v;
    // u moved after v
    if ((mask & 1u) && Urem1 < (kBig >> 1)) {
        int dl = Urem1 + VK1 + t00 + t01 + wL * max(VLQ + Ud, 0);
        if (TW) {
            const int a1 = Vtau + t00, w1 = max(a1 - Ul, 0);
            const int a2 = max(a1, Ue) - w1 + Us + t01, w2 = max(a2 - VLg, 0);
            dl += wT * (w1 + w2);
        }
        evaluated |= 1u;
        TGA_TRY(dl, au * W + av);
    }
    // the runs of 2 and 3 starting at u moved after v
    if (OR) {
        const int UC2 = u3.x, Uld2 = u3.y, UC3 = u3.z, Uld3 = u3.w;
        if (UC2 < (kBig >> 1)) {
            int dl = UC2 + VK1 + t00 + t11 + wL * max(VLQ + Uld2, 0);
            if (TW) {
                const int UE2 = u5.z, UL2 = u5.w, UDm2 = u6.x;
                const int a1 = Vtau + t00, w1 = max(a1 - UL2, 0);
                const int a2 = max(a1, UE2) - w1 + UDm2 + t11, w2 = max(a2 - VLg, 0);
                dl += wT * (w1 + w2);
            }
            evaluated |= 16u;
            TGA_TRY(dl, 4u * W2 + au * W + av);
        }
        if (UC3 < (kBig >> 1)) {
            int dl = UC3 + VK1 + t00 + t21 + wL * max(VLQ + Uld3, 0);
            if (TW) {
                const int UE3 = u6.y, UL3 = u6.z, UDm3 = u6.w;
                const int a1 = Vtau + t00, w1 = max(a1 - UL3, 0);
                const int a2 = max(a1, UE3) - w1 + UDm3 + t21, w2 = max(a2 - VLg, 0);
                dl += wT * (w1 + w2);
            }
            evaluated |= 32u;
            TGA_TRY(dl, 5u * W2 + au * W + av);
        }
    }
    // swap u <-> v
    if ((mask & 2u) && vcust && pair_once) {
        int dl = UK2 + VK2 + tm10 + t10 + t0m1 + t01 + wL * (max(ULQd + Vd, 0) + max(VLQd + Ud, 0));
        if (TW) {
            const int a1 = UtauP + tm10, w1 = max(a1 - Vl, 0);
            const int a2 = max(a1, Ve) - w1 + Vs + t10, w2 = max(a2 - ULg, 0);
            const int b1 = VtauP + t0m1, x1 = max(b1 - Ul, 0);
            const int b2 = max(b1, Ue) - x1 + Us + t01, x2 = max(b2 - VLg, 0);
            dl += wT * (w1 + w2 + x1 + x2);
        }
        evaluated |= 2u;
        TGA_TRY(dl, W2 + min(au, av) * W + max(au, av));
    }
    // 2-opt*: head(u) + tail after v, head(v) + tail after u
    if ((mask & 8u) && (pair_once || !vcust)) {
        int dl = UFc + VGc + VFc + UGc + t01 + t10 + wL * (max(Uloadf + VloadgQ, 0) + max(Vloadf + UloadgQ, 0));
        if (TW) dl += wT * (max(Utau + t01 - VLg, 0) + max(Vtau + t10 - ULg, 0));
        evaluated |= 8u;
        TGA_TRY(dl, 3u * W2 + (Uroute < Vroute ? au * W + av : av * W + au));
    }
    return evaluated;
}

// ---------------------------------------------------------------------------
// intra-route evaluation
//
// Sweeps over a route (the batched kernel's intra-route evaluation, and the
// fallback for time-window routes too long for the subsequence tables).
// One warp per route.  The route's elements (0 = start depot, 1..L
// customers, L+1 = end depot) are staged in shared memory with their node
// data, the prefix/suffix attributes of every anchor, and -- when it fits --
// the route's (L+2) x (L+2) distance block, read as contiguous row segments
// of the position-ordered distance copy.  Lane i then sweeps the other end
// of every move that starts (or ends) at element i, maintaining the middle
// segment incrementally with the concatenation operator, so each candidate
// is O(1) (route-based extraction of Section 5.3.1 with the attribute-matrix
// rows of Section 4.2 built on the fly).

constexpr int kIntraWarps = 4;
constexpr int kIntraSmemPerWarp = 2816;      // ints (11 KB)

struct RouteView {
    const Dev *d;
    int r, L, E, st;
    bool inS;                 // distance block in shared memory
    const int *node, *e, *l, *s, *tau, *twf, *distf, *Lg, *twg, *distg;
    // pickups: prefix L_I, L_O, L_M through element k; suffix L_I, L_M after it
    const int *lif, *lof, *lmf, *lig, *lmg;
    const int *D;             // E x E (if inS)
    // loads of the customer at element k (1..L)
    __device__ __forceinline__ Ld ldn(int k) const {
        Ld x;
        x.i = lif[k] - lif[k - 1];
        x.o = lof[k] - lof[k - 1];
        x.m = max(x.i, x.o);
        return x;
    }
    __device__ __forceinline__ int c(int a, int b) const {
        if (inS) return D[a * E + b];
        return TGA_LDG(d->pcol + (size_t)node[a] * d->ldp + kColOff + st + b);
    }
    __device__ __forceinline__ int anchor(int k) const { return k == 0 ? d->n + 1 + r : node[k]; }
    __device__ __forceinline__ Seg seg(int k, int out) const {
        Seg x;
        x.E = e[k]; x.L = l[k]; x.D = s[k]; x.TW = 0; x.dist = 0; x.load = 0; x.out = out;
        return x;
    }
};

// kinds selects the sweeps this call runs: bit k-1 forward relocate/or-opt
// of a run of k, bit 3 swap, bit 4 2-opt, bit 4+k backward run of k, bit 8
// the swaps of runs (XS).
// PD: pickups; each candidate adds the change of the load excess of the
// route's largest load (basePen = the current excess), built by the same
// incremental concatenations with the loads of Section 4.3.2.
template <bool TW, bool PD = false, bool XS = false>
__device__ void intra_anchor(const RouteView &V, int i, unsigned mask, int wT, int baseDist, int baseTw,
                             unsigned W, unsigned W2, int &best, unsigned &bidx, unsigned kinds = 0xffu,
                             int Q = 0, int wL = 0, int basePen = 0) {
    const int L = V.L;
    // load term of a new route whose largest load is LM
    auto pen = [&](int LM) { return wL * (max(LM - Q, 0) - basePen); };
    if (i >= 1) {
        // ---------------- moves that take the customer at element i forward
        const unsigned xi = (unsigned)V.node[i];
        const int ptau = V.tau[i - 1], ptwf = V.twf[i - 1], pdist = V.distf[i - 1];
        // relocate / or-opt of the run i..i+k-1 to after element j, j >= i+k
        for (int k = 1; k <= 3; ++k) {
            const int op = k == 1 ? 0 : k + 2;
            if (!(kinds & (1u << (k - 1))) || !(mask & (1u << op)) || i + k - 1 > L) continue;
            Seg run = V.seg(i, V.c(i, i + 1));
            for (int t = 1; t < k; ++t) run = seg_cat(run, V.seg(i + t, V.c(i + t, i + t + 1)));
            Ld runl{0, 0, 0};
            int ao = 0, am = 0;                  // prefix through i-1, then the elements i+k..j
            if (PD) {
                runl = V.ldn(i);
                for (int t = 1; t < k; ++t) runl = ld_cat(runl, V.ldn(i + t));
                ao = V.lof[i - 1]; am = V.lmf[i - 1];
            }
            int tau = ptau, tw = ptwf, dist = pdist, last = i - 1;
            for (int j = i + k; j <= L; ++j) {
                const int c1 = V.c(last, j);
                dist += c1;
                if (TW) {
                    const int a = tau + c1;
                    const int w = max(a - V.l[j], 0);
                    tau = max(a, V.e[j]) - w + V.s[j];
                    tw += w;
                }
                last = j;
                const int cA = V.c(j, i), cB = V.c(i + k - 1, j + 1);
                int delta = dist + cA + run.dist + cB + V.distg[j] - baseDist;
                if (TW) {
                    const int a1 = tau + cA, w1 = max(a1 - run.L, 0);
                    const int a2 = max(a1, run.E) - w1 + run.D - run.TW + cB;
                    const int w2 = max(a2 - V.Lg[j], 0);
                    delta += wT * (tw + w1 + run.TW + w2 + V.twg[j] - baseTw);
                }
                if (PD) {
                    const Ld nj = V.ldn(j);
                    am = max(am + nj.i, ao + nj.m);
                    ao += nj.o;
                    delta += pen(ld_close(ao, am, runl, V.lig[j], V.lmg[j]));
                }
                TGA_TRY(delta, (unsigned)op * W2 + xi * W + (unsigned)V.node[j]);
            }
        }
        // swap element i <-> element j, j > i
        if ((kinds & 8u) && (mask & 2u)) {
            Seg M{};
            Ld Ml{0, 0, 0};
            for (int j = i + 1; j <= L; ++j) {
                if (j > i + 2) M = seg_cat(M, V.seg(j - 1, V.c(j - 1, j)));
                else if (j == i + 2) M = V.seg(i + 1, V.c(i + 1, j));
                if (PD && j >= i + 2) Ml = j == i + 2 ? V.ldn(i + 1) : ld_cat(Ml, V.ldn(j - 1));
                const bool hasM = j > i + 1;
                const int ca = V.c(i - 1, j);
                int dist = pdist + ca + V.distg[j];
                int tau = 0, tw = 0;
                if (TW) {
                    const int a = ptau + ca, w = max(a - V.l[j], 0);
                    tau = max(a, V.e[j]) - w + V.s[j];
                    tw = ptwf + w;
                }
                int last = j;
                if (hasM) {
                    const int cb = V.c(j, i + 1);
                    dist += cb + M.dist;
                    if (TW) {
                        const int a = tau + cb, w = max(a - M.L, 0);
                        tau = max(a, M.E) - w + M.D - M.TW;
                        tw += w + M.TW;
                    }
                    last = j - 1;
                }
                const int cc = V.c(last, i), cd = V.c(i, j + 1);
                dist += cc + cd;
                int delta = dist - baseDist;
                if (TW) {
                    const int a = tau + cc, w = max(a - V.l[i], 0);
                    const int t2 = max(a, V.e[i]) - w + V.s[i];
                    const int w4 = max(t2 + cd - V.Lg[j], 0);
                    delta += wT * (tw + w + w4 + V.twg[j] - baseTw);
                }
                if (PD) {   // prefix(i-1) + x_j + (i+1..j-1) + x_i + suffix(j)
                    Ld g = V.ldn(j);
                    if (hasM) g = ld_cat(g, Ml);
                    g = ld_cat(g, V.ldn(i));
                    delta += pen(ld_close(V.lof[i - 1], V.lmf[i - 1], g, V.lig[j], V.lmg[j]));
                }
                const unsigned xj = (unsigned)V.node[j];
                TGA_TRY(delta, W2 + min(xi, xj) * W + max(xi, xj));
            }
        }
        // 2-opt: reverse elements i..j, j > i
        if ((kinds & 16u) && (mask & 4u)) {
            Seg Rv = V.seg(i, 0);
            Ld Rl{0, 0, 0};
            if (PD) Rl = V.ldn(i);
            for (int j = i + 1; j <= L; ++j) {
                Rv = seg_cat(V.seg(j, V.c(j, j - 1)), Rv);
                const int ca = V.c(i - 1, j), cb = V.c(i, j + 1);
                int delta = pdist + ca + Rv.dist + cb + V.distg[j] - baseDist;
                if (TW) {
                    const int a1 = ptau + ca, w1 = max(a1 - Rv.L, 0);
                    const int a2 = max(a1, Rv.E) - w1 + Rv.D - Rv.TW + cb;
                    const int w2 = max(a2 - V.Lg[j], 0);
                    delta += wT * (ptwf + w1 + Rv.TW + w2 + V.twg[j] - baseTw);
                }
                if (PD) {   // prefix(i-1) + reversed (i..j) + suffix(j)
                    Rl = ld_cat(V.ldn(j), Rl);
                    delta += pen(ld_close(V.lof[i - 1], V.lmf[i - 1], Rl, V.lig[j], V.lmg[j]));
                }
                TGA_TRY(delta, 2u * W2 + xi * W + (unsigned)V.node[j]);
            }
        }
    }
    // ---------------- swaps of runs starting at element i: the run
    // i..i+kx-1 exchanges places with a later run y..y+ky-1 (y >= i+kx);
    // the middle i+kx..y-1 grows with y
    if (XS && (kinds & 256u) && i >= 1) {
        auto enter = [&](int t, const Seg &g, int &warp) {
            const int w = max(t - g.L, 0);
            warp += w + g.TW;
            return max(t, g.E) - w + g.D - g.TW;
        };
        const unsigned xi = (unsigned)V.node[i];
        for (int v = 0; v < 3; ++v) {
            const int kx = v == 0 ? 1 : 2, ky = v == 1 ? 1 : 2;
            const unsigned op = (kx == 2 && ky == 2) ? 7u : 6u;
            if (!(mask & (1u << op)) || i + kx - 1 > L) continue;
            Seg rx = V.seg(i, V.c(i, i + 1));
            if (kx == 2) rx = seg_cat(rx, V.seg(i + 1, 0));
            Seg M{};
            for (int y = i + kx; y + ky - 1 <= L; ++y) {
                if (y == i + kx + 1) M = V.seg(i + kx, V.c(i + kx, y));
                else if (y > i + kx + 1) M = seg_cat(M, V.seg(y - 1, V.c(y - 1, y)));
                const bool hasM = y > i + kx;
                const int last = y + ky - 1, xe = i + kx - 1;
                Seg ry = V.seg(y, V.c(y, y + 1));
                if (ky == 2) ry = seg_cat(ry, V.seg(y + 1, 0));
                const int c1 = V.c(i - 1, y), c2 = V.c(last, hasM ? i + kx : i);
                const int c4 = V.c(xe, last + 1);
                int dist = V.distf[i - 1] + c1 + ry.dist + c2 + rx.dist + c4 + V.distg[last];
                int c3 = 0;
                if (hasM) {
                    c3 = V.c(y - 1, i);
                    dist += M.dist + c3;
                }
                int delta = dist - baseDist;
                if (TW) {
                    int warp = V.twf[i - 1];
                    int t = enter(V.tau[i - 1] + c1, ry, warp);
                    if (hasM) t = enter(t + c2, M, warp) + c3;
                    else t += c2;
                    t = enter(t, rx, warp);
                    const int w4 = max(t + c4 - V.Lg[last], 0);
                    delta += wT * (warp + w4 + V.twg[last] - baseTw);
                }
                const unsigned xy = (unsigned)V.node[y];
                const unsigned a = kx == ky ? min(xi, xy) : (kx == 1 ? xi : xy);
                const unsigned b = kx == ky ? max(xi, xy) : (kx == 1 ? xy : xi);
                TGA_TRY(delta, op * W2 + a * W + b);
            }
        }
    }
    // ---------------- moves whose destination is element j = i: the run
    // t..t+k-1, t >= j+2, moves back to just after element j.
    const int j = i;
    const unsigned aj = (unsigned)V.anchor(j);
    for (int k = 1; k <= 3; ++k) {
        const int op = k == 1 ? 0 : k + 2;
        if (!(kinds & (1u << (4 + k))) || !(mask & (1u << op)) || j + 2 + k - 1 > L) continue;
        Seg M = V.seg(j + 1, V.c(j + 1, j + 2));
        Ld Ml{0, 0, 0};
        if (PD) Ml = V.ldn(j + 1);
        for (int t = j + 2; t + k - 1 <= L; ++t) {
            if (t > j + 2) M = seg_cat(M, V.seg(t - 1, V.c(t - 1, t)));
            if (PD && t > j + 2) Ml = ld_cat(Ml, V.ldn(t - 1));
            Seg run = V.seg(t, V.c(t, t + 1));
            for (int u = 1; u < k; ++u) run = seg_cat(run, V.seg(t + u, V.c(t + u, t + u + 1)));
            const int w = t + k - 1;
            const int ca = V.c(j, t), cb = V.c(w, j + 1), cc = V.c(t - 1, t + k);
            int delta = V.distf[j] + ca + run.dist + cb + M.dist + cc + V.distg[w] - baseDist;
            if (TW) {
                const int a1 = V.tau[j] + ca, w1 = max(a1 - run.L, 0);
                const int a2 = max(a1, run.E) - w1 + run.D - run.TW + cb;
                const int w2 = max(a2 - M.L, 0);
                const int a3 = max(a2, M.E) - w2 + M.D - M.TW + cc;
                const int w3 = max(a3 - V.Lg[w], 0);
                delta += wT * (V.twf[j] + w1 + run.TW + w2 + M.TW + w3 + V.twg[w] - baseTw);
            }
            if (PD) {   // prefix(j) + run (t..w) + (j+1..t-1) + suffix(w)
                Ld g = V.ldn(t);
                for (int u = 1; u < k; ++u) g = ld_cat(g, V.ldn(t + u));
                g = ld_cat(g, Ml);
                delta += pen(ld_close(V.lof[j], V.lmf[j], g, V.lig[w], V.lmg[w]));
            }
            TGA_TRY(delta, (unsigned)op * W2 + (unsigned)V.node[t] * W + aj);
        }
    }
}

// Intra-route candidates of route r with one warp (all 32 lanes call);
// S is this warp's kIntraSmemPerWarp ints of shared memory.
template <bool TW, bool PD = false, bool XS = false>
__device__ void intra_route(const Dev &d, int r, int lane, int *S, int &best, unsigned &bidx) {
    const RouteRec R = d.rrec[TGA_IX(r, d.m)];
    const int L = R.len;
    if (L < 2) return;
    RouteView V;
    V.d = &d; V.r = r; V.L = L; V.E = L + 2; V.st = R.start;
    const int E = V.E;
    constexpr int NV = PD ? kIntraVecPD : kIntraVec;
    const bool vecS = NV * E <= kIntraSmemPerWarp;
    V.inS = vecS && NV * E + E * E <= kIntraSmemPerWarp;
    // per-element arrays: shared memory when they fit, else this
    // route's own slice [start+r, start+r+E) of the global scratch
    int *base = vecS ? S : d.scr_intra + (R.start + r);
    const int stride = vecS ? E : d.Wp + d.m;
    int *node = base, *e = base + stride, *l = base + 2 * stride, *s = base + 3 * stride;
    int *tau = base + 4 * stride, *twf = base + 5 * stride, *distf = base + 6 * stride;
    int *Lg = base + 7 * stride, *twg = base + 8 * stride, *distg = base + 9 * stride;
    V.node = node; V.e = e; V.l = l; V.s = s; V.tau = tau; V.twf = twf; V.distf = distf;
    V.Lg = Lg; V.twg = twg; V.distg = distg;
    int *lif = base + 10 * stride, *lof = base + 11 * stride, *lmf = base + 12 * stride;
    int *lig = base + 13 * stride, *lmg = base + 14 * stride;
    V.lif = lif; V.lof = lof; V.lmf = lmf; V.lig = lig; V.lmg = lmg;
    for (int k = lane; k < E; k += 32) {
        const int a = (k == 0) ? d.n + 1 + r : (k <= L ? d.seq[TGA_IX(V.st + k, d.Wp)] : -1);
        const int x = (k >= 1 && k <= L) ? a : 0;
        node[k] = x;
        if (TW) { e[k] = __ldg(d.early + x); l[k] = __ldg(d.late + x); s[k] = __ldg(d.service + x); }
        else { e[k] = 0; l[k] = 0; s[k] = 0; }
        if (a >= 0) {
            const BRec b = d.brec[TGA_IX(a, d.W + 1)];
            tau[k] = b.tau; twf[k] = b.twf; distf[k] = b.distf;
            Lg[k] = b.Lg; twg[k] = b.twg; distg[k] = b.distg;
            if (PD) { lif[k] = b.loadf; lof[k] = b.lof; lmf[k] = b.lmf; lig[k] = b.loadg; lmg[k] = b.lmg; }
        } else {
            tau[k] = 0; twf[k] = 0; distf[k] = 0; Lg[k] = 0; twg[k] = 0; distg[k] = 0;
            if (PD) { lif[k] = 0; lof[k] = 0; lmf[k] = 0; lig[k] = 0; lmg[k] = 0; }
        }
    }
    __syncwarp();
    if (V.inS) {
        int *D = S + NV * E;
        for (int t = lane; t < E * E; t += 32) {
            const int a = t / E, b = t - a * E;
            D[t] = d.pcol[(size_t)TGA_IX(node[a], d.n + 1) * d.ldp + TGA_IX(kColOff + V.st + b, d.ldp)];
        }
        V.D = D;
    } else {
        V.D = nullptr;
    }
    __syncwarp();
    const unsigned W = (unsigned)d.W, W2 = W * W;
    const int wT = TW ? d.wT : 0;
    for (int i = lane; i <= L; i += 32)
        intra_anchor<TW, PD, XS>(V, i, d.op_mask, wT, R.dist, R.tw, W, W2, best, bidx, 0x1ffu, d.Q, d.wL,
                              max(R.lm - d.Q, 0));
    __syncwarp();
}

// Intra-route candidates of route r with a whole block: all warps stage the
// route into S (kIntraSmemPerWarp ints), then warp w runs the sweep kinds
// {w, w+nw, ...} of every anchor, so the serial sweeps of one anchor are
// spread over the warps.
template <bool TW, bool PD = false, bool XS = false>
__device__ void intra_route_block(const Dev &d, int r, int *S, int &best, unsigned &bidx) {
    const RouteRec R = d.rrec[TGA_IX(r, d.m)];
    const int L = R.len;
    if (L < 2) return;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    RouteView V;
    V.d = &d; V.r = r; V.L = L; V.E = L + 2; V.st = R.start;
    const int E = V.E;
    constexpr int NV = PD ? kIntraVecPD : kIntraVec;
    const bool vecS = NV * E <= kIntraSmemPerWarp;
    V.inS = vecS && NV * E + E * E <= kIntraSmemPerWarp;
    int *base = vecS ? S : d.scr_intra + (R.start + r);
    const int stride = vecS ? E : d.Wp + d.m;
    int *node = base, *e = base + stride, *l = base + 2 * stride, *s = base + 3 * stride;
    int *tau = base + 4 * stride, *twf = base + 5 * stride, *distf = base + 6 * stride;
    int *Lg = base + 7 * stride, *twg = base + 8 * stride, *distg = base + 9 * stride;
    V.node = node; V.e = e; V.l = l; V.s = s; V.tau = tau; V.twf = twf; V.distf = distf;
    V.Lg = Lg; V.twg = twg; V.distg = distg;
    int *lif = base + 10 * stride, *lof = base + 11 * stride, *lmf = base + 12 * stride;
    int *lig = base + 13 * stride, *lmg = base + 14 * stride;
    V.lif = lif; V.lof = lof; V.lmf = lmf; V.lig = lig; V.lmg = lmg;
    for (int k = tid; k < E; k += nthr) {
        const int a = (k == 0) ? d.n + 1 + r : (k <= L ? d.seq[TGA_IX(V.st + k, d.Wp)] : -1);
        const int x = (k >= 1 && k <= L) ? a : 0;
        node[k] = x;
        if (TW) { e[k] = __ldg(d.early + x); l[k] = __ldg(d.late + x); s[k] = __ldg(d.service + x); }
        else { e[k] = 0; l[k] = 0; s[k] = 0; }
        if (a >= 0) {
            const BRec b = d.brec[TGA_IX(a, d.W + 1)];
            tau[k] = b.tau; twf[k] = b.twf; distf[k] = b.distf;
            Lg[k] = b.Lg; twg[k] = b.twg; distg[k] = b.distg;
            if (PD) { lif[k] = b.loadf; lof[k] = b.lof; lmf[k] = b.lmf; lig[k] = b.loadg; lmg[k] = b.lmg; }
        } else {
            tau[k] = 0; twf[k] = 0; distf[k] = 0; Lg[k] = 0; twg[k] = 0; distg[k] = 0;
            if (PD) { lif[k] = 0; lof[k] = 0; lmf[k] = 0; lig[k] = 0; lmg[k] = 0; }
        }
    }
    __syncthreads();
    if (V.inS) {
        int *D = S + NV * E;
        for (int t = tid; t < E * E; t += nthr) {
            const int a = t / E, b = t - a * E;
            D[t] = d.pcol[(size_t)TGA_IX(node[a], d.n + 1) * d.ldp + TGA_IX(kColOff + V.st + b, d.ldp)];
        }
        V.D = D;
    } else {
        V.D = nullptr;
    }
    __syncthreads();
    unsigned kinds = 0;
    for (int k = warp; k < (XS ? 9 : 8); k += nw) kinds |= 1u << k;
    const unsigned W = (unsigned)d.W, W2 = W * W;
    const int wT = TW ? d.wT : 0;
    for (int i = lane; i <= L; i += 32)
        intra_anchor<TW, PD, XS>(V, i, d.op_mask, wT, R.dist, R.tw, W, W2, best, bidx, kinds, d.Q, d.wL,
                              max(R.lm - d.Q, 0));
}

// ---------------------------------------------------------------------------
// Intra-route candidates of a time-window route from subsequence tables.
//
// The route's attribute matrix of Section 4.2 -- the time-window data
// (E, L, D - T_V, T_V) of every subsequence x_i..x_j of customers, forward
// (F) and reversed (R, for 2-opt) -- is built in shared memory, one thread
// per row i extending its row by the concatenation operator of Section 4.3.
// Every intra-route candidate is then an O(1) concatenation of the prefix
// before the move, at most three table entries or single customers, and the
// suffix after it (route-based extraction, Section 5.3.1), so the threads of
// the block take the (i, j) pairs of the route independently: the critical
// path is one row of the table instead of a sweep per anchor.  Routes longer
// than kTabMaxL customers fall back to intra_route_block.

constexpr int kTabMaxL = 40;
constexpr int kTabEntries = kTabMaxL * (kTabMaxL + 1) / 2;
// shared ints: per-element arrays, the distance block and both int4 tables;
// with pickups also five load arrays and the forward and reversed L_M tables
constexpr int kIntraTabSmemInts =
    ((kIntraVec * (kTabMaxL + 2) + (kTabMaxL + 2) * (kTabMaxL + 2) + 3) / 4) * 4 + 2 * 4 * kTabEntries;
constexpr int kIntraTabSmemIntsPD = kIntraTabSmemInts + 5 * (kTabMaxL + 2) + 2 * kTabEntries;

// Entry (i, j), 1 <= i <= j <= L, of a packed upper-triangular table.
__device__ __forceinline__ int tri_at(int i, int j, int L) {
    return (i - 1) * L - ((i - 1) * (i - 2)) / 2 + (j - i);
}

// a (+) b for time-window data {E, L, D - T_V, T_V} with travel time t
// between them (the concatenation of Section 4.3 in the difference form).
__device__ __forceinline__ int4 tw_cat(const int4 a, const int4 b, int t) {
    const int dt = a.z + t;
    const int dw = max(b.x - dt - a.y, 0);
    const int dv = max(a.x + dt - b.y, 0);
    return make_int4(max(b.x - dt, a.x) - dw, min(b.y - dt, a.y) + dv, a.z + t + dw - dv + b.z, a.w + dv + b.w);
}

// Departure time and warp after entering segment g at arrival time a.
__device__ __forceinline__ int tw_enter(int a, const int4 g, int &warp) {
    const int w = max(a - g.y, 0);
    warp += w + g.w;
    return max(a, g.x) - w + g.z;
}

// XS: also the swaps of runs inside the route (op ranks 6, 7).
template <bool PD = false, bool XS = false>
__device__ void intra_route_table(const Dev &d, int r, int *S, int &best, unsigned &bidx) {
    const RouteRec R = d.rrec[TGA_IX(r, d.m)];
    const int L = R.len;
    if (L < 2) return;
    if (L > kTabMaxL) {
        intra_route_block<true, PD, XS>(d, r, S, best, bidx);
        return;
    }
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int E = L + 2, st = R.start;
    int *node = S, *e = S + E, *l = S + 2 * E, *s = S + 3 * E, *tau = S + 4 * E, *twf = S + 5 * E;
    int *distf = S + 6 * E, *Lg = S + 7 * E, *twg = S + 8 * E, *distg = S + 9 * E;
    int *D = S + kIntraVec * E;                                   // E x E distances
    int4 *Ft = reinterpret_cast<int4 *>(S + ((kIntraVec * E + E * E + 3) / 4) * 4);
    int4 *Rt = Ft + L * (L + 1) / 2;
    // pickups: prefix L_I, L_O, L_M through element k, suffix L_I, L_M after
    // it, and the L_M of every subsequence forward (FtM) and reversed (RtM)
    int *lif = reinterpret_cast<int *>(Rt + L * (L + 1) / 2);
    int *lof = lif + E, *lmf = lif + 2 * E, *lig = lif + 3 * E, *lmg = lif + 4 * E;
    int *FtM = lif + 5 * E, *RtM = FtM + L * (L + 1) / 2;
    // ---- staging: element records, and the distance block from the
    // position-ordered copy (row of element a, columns st .. st+E-1), both
    // issued right after the positions are known
    for (int k = tid; k < E; k += nthr) {
        const int a = (k == 0) ? d.n + 1 + r : (k <= L ? d.seq[TGA_IX(st + k, d.Wp)] : -1);
        const int x = (k >= 1 && k <= L) ? a : 0;
        node[k] = x;
        e[k] = __ldg(d.early + x); l[k] = __ldg(d.late + x); s[k] = __ldg(d.service + x);
        if (a >= 0) {
            const BRec b = d.brec[TGA_IX(a, d.W + 1)];
            tau[k] = b.tau; twf[k] = b.twf; distf[k] = b.distf;
            Lg[k] = b.Lg; twg[k] = b.twg; distg[k] = b.distg;
            if (PD) { lif[k] = b.loadf; lof[k] = b.lof; lmf[k] = b.lmf; lig[k] = b.loadg; lmg[k] = b.lmg; }
        } else {
            tau[k] = 0; twf[k] = 0; distf[k] = 0; Lg[k] = 0; twg[k] = 0; distg[k] = 0;
            if (PD) { lif[k] = 0; lof[k] = 0; lmf[k] = 0; lig[k] = 0; lmg[k] = 0; }
        }
    }
#pragma unroll 4
    for (int t = tid; t < E * E; t += nthr) {
        const int a = t / E, b = t - a * E;
        const int x = (a >= 1 && a <= L) ? d.seq[TGA_IX(st + a, d.Wp)] : 0;
        D[t] = TGA_LDG(d.pcol + (size_t)TGA_IX(x, d.n + 1) * d.ldp + TGA_IX(kColOff + st + b, d.ldp));
    }
    __syncthreads();
    // ---- tables: thread c < L extends forward row i = c+1, thread L + c the
    // reversed row (x_j .. x_i, entered from x_j)
    for (int c = tid; c < 2 * L; c += nthr) {
        const bool rev = c >= L;
        const int i = (rev ? c - L : c) + 1;
        int4 *T = rev ? Rt : Ft;
        int4 cur = make_int4(e[i], l[i], s[i], 0);
        T[tri_at(i, i, L)] = cur;
        for (int j = i + 1; j <= L; ++j) {
            const int4 nx = make_int4(e[j], l[j], s[j], 0);
            cur = rev ? tw_cat(nx, cur, D[j * E + j - 1]) : tw_cat(cur, nx, D[(j - 1) * E + j]);
            T[tri_at(i, j, L)] = cur;
        }
        if (PD) {
            int *TM = rev ? RtM : FtM;
            auto nodeld = [&](int k) {
                Ld x;
                x.i = lif[k] - lif[k - 1]; x.o = lof[k] - lof[k - 1]; x.m = max(x.i, x.o);
                return x;
            };
            Ld cl = nodeld(i);
            TM[tri_at(i, i, L)] = cl.m;
            for (int j = i + 1; j <= L; ++j) {
                cl = rev ? ld_cat(nodeld(j), cl) : ld_cat(cl, nodeld(j));
                TM[tri_at(i, j, L)] = cl.m;
            }
        }
    }
    __syncthreads();
    // loads of the subsequence x_i..x_j (forward, or reversed when rev)
    auto segld = [&](int i, int j, bool rev) {
        Ld x;
        x.i = lif[j] - lif[i - 1]; x.o = lof[j] - lof[i - 1];
        x.m = (rev ? RtM : FtM)[tri_at(i, j, L)];
        return x;
    };
    const int Q = d.Q, wL = d.wL, basePen = PD ? max(R.lm - Q, 0) : 0;
    auto pen = [&](int LM) { return wL * (max(LM - Q, 0) - basePen); };
    // ---- candidates: pair (i, j), 0 <= i < j <= L, one pair per thread
    const unsigned mask = d.op_mask;
    const unsigned W = (unsigned)d.W, W2 = W * W;
    const int wT = d.wT, baseDist = R.dist, baseTw = R.tw;
    // exchange of the run x..x+kx-1 with the later run y..y+ky-1 (x + kx <= y):
    // prefix(x-1) + (y..) + (x+kx..y-1) + (x..) + suffix(y+ky-1)
    auto xchg = [&](int x, int kx, int y, int ky) {
        const int last = y + ky - 1, xe = x + kx - 1;
        const int c1 = D[(x - 1) * E + y];
        int tw = twf[x - 1];
        int tx = tw_enter(tau[x - 1] + c1, Ft[tri_at(y, last, L)], tw);
        int dist = distf[x - 1] + c1 + (distf[last] - distf[y]);
        int prev = last;
        if (y > x + kx) {
            const int c2 = D[last * E + x + kx];
            tx = tw_enter(tx + c2, Ft[tri_at(x + kx, y - 1, L)], tw);
            dist += c2 + (distf[y - 1] - distf[x + kx]);
            prev = y - 1;
        }
        const int c3 = D[prev * E + x];
        tx = tw_enter(tx + c3, Ft[tri_at(x, xe, L)], tw);
        const int c4 = D[xe * E + last + 1];
        const int w4 = max(tx + c4 - Lg[last], 0);
        dist += c3 + (distf[xe] - distf[x]) + c4 + distg[last];
        return dist - baseDist + wT * (tw + w4 + twg[last] - baseTw);
    };
    const int L1 = L + 1;
    const unsigned adep = (unsigned)(d.n + 1 + r);
    for (int t = tid; t < L1 * L1; t += nthr) {
        const int i = t / L1, j = t - i * L1;
        if (j <= i) continue;
        if (i >= 1) {
            const unsigned xi = (unsigned)node[i], xj = (unsigned)node[j];
            const int ptau = tau[i - 1], ptwf = twf[i - 1], pdist = distf[i - 1];
            // relocate (k = 1) / or-opt (k = 2, 3): run x_i..x_{i+k-1} to
            // just after x_j, j >= i+k: prefix(i-1) + (i+k..j) + run + suffix(j)
#pragma unroll
            for (int k = 1; k <= 3; ++k) {
                const int op = k == 1 ? 0 : k + 2;
                if (!(mask & (1u << op)) || j < i + k) continue;
                const int c0 = D[(i - 1) * E + i + k];
                int tw = ptwf;
                const int tm = tw_enter(ptau + c0, Ft[tri_at(i + k, j, L)], tw);
                const int cA = D[j * E + i], cB = D[(i + k - 1) * E + j + 1];
                const int tr = tw_enter(tm + cA, Ft[tri_at(i, i + k - 1, L)], tw);
                const int w2 = max(tr + cB - Lg[j], 0);
                const int dist = pdist + c0 + (distf[j] - distf[i + k]) + cA + (distf[i + k - 1] - distf[i]) + cB +
                                 distg[j];
                int lp = 0;
                if (PD) {   // prefix(i-1) + (i+k..j) + run + suffix(j)
                    const Ld g = ld_cat(segld(i + k, j, false), segld(i, i + k - 1, false));
                    lp = pen(ld_close(lof[i - 1], lmf[i - 1], g, lig[j], lmg[j]));
                }
                TGA_TRY(dist - baseDist + wT * (tw + w2 + twg[j] - baseTw) + lp, (unsigned)op * W2 + xi * W + xj);
            }
            // swap x_i <-> x_j
            if (mask & 2u) {
                const int ca = D[(i - 1) * E + j];
                int tw = ptwf;
                int tx = tw_enter(ptau + ca, make_int4(e[j], l[j], s[j], 0), tw);
                int dist = pdist + ca + distg[j];
                int last = j;
                if (j > i + 1) {
                    const int cb = D[j * E + i + 1];
                    tx = tw_enter(tx + cb, Ft[tri_at(i + 1, j - 1, L)], tw);
                    dist += cb + (distf[j - 1] - distf[i + 1]);
                    last = j - 1;
                }
                const int cc = D[last * E + i], cd = D[i * E + j + 1];
                tx = tw_enter(tx + cc, make_int4(e[i], l[i], s[i], 0), tw);
                const int w4 = max(tx + cd - Lg[j], 0);
                int lp = 0;
                if (PD) {   // prefix(i-1) + x_j + (i+1..j-1) + x_i + suffix(j)
                    Ld g = segld(j, j, false);
                    if (j > i + 1) g = ld_cat(g, segld(i + 1, j - 1, false));
                    g = ld_cat(g, segld(i, i, false));
                    lp = pen(ld_close(lof[i - 1], lmf[i - 1], g, lig[j], lmg[j]));
                }
                TGA_TRY(dist + cc + cd - baseDist + wT * (tw + w4 + twg[j] - baseTw) + lp,
                        W2 + min(xi, xj) * W + max(xi, xj));
            }
            if (XS) {
                // a customer with a run of two, and two runs of two
                if ((mask & 64u) && j + 1 <= L)          // x_i alone, the run x_j x_j+1
                    TGA_TRY(xchg(i, 1, j, 2), 6u * W2 + xi * W + xj);
                if ((mask & 64u) && i + 1 <= L && j >= i + 2)   // the run x_i x_i+1, x_j alone
                    TGA_TRY(xchg(i, 2, j, 1), 6u * W2 + xj * W + xi);
                if ((mask & 128u) && j >= i + 2 && j + 1 <= L)
                    TGA_TRY(xchg(i, 2, j, 2), 7u * W2 + min(xi, xj) * W + max(xi, xj));
            }
            // 2-opt: reverse x_i..x_j
            if (mask & 4u) {
                const int ca = D[(i - 1) * E + j], cb = D[i * E + j + 1];
                int tw = ptwf;
                const int tx = tw_enter(ptau + ca, Rt[tri_at(i, j, L)], tw);
                const int w2 = max(tx + cb - Lg[j], 0);
                const int lp = PD ? pen(ld_close(lof[i - 1], lmf[i - 1], segld(i, j, true), lig[j], lmg[j])) : 0;
                TGA_TRY(pdist + ca + (distf[j] - distf[i]) + cb + distg[j] - baseDist +
                            wT * (tw + w2 + twg[j] - baseTw) + lp,
                        2u * W2 + xi * W + xj);
            }
        }
        // the run x_j..x_{j+k-1} moves back to just after element i (j >= i+2):
        // prefix(i) + run + (i+1..j-1) + suffix(j+k-1)
        const unsigned ai = i == 0 ? adep : (unsigned)node[i];
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            const int op = k == 1 ? 0 : k + 2;
            const int w = j + k - 1;
            if (!(mask & (1u << op)) || j < i + 2 || w > L) continue;
            const int ca = D[i * E + j], cb = D[w * E + i + 1], cc = D[(j - 1) * E + j + k];
            int tw = twf[i];
            int tx = tw_enter(tau[i] + ca, Ft[tri_at(j, w, L)], tw);
            tx = tw_enter(tx + cb, Ft[tri_at(i + 1, j - 1, L)], tw);
            const int w3 = max(tx + cc - Lg[w], 0);
            const int dist = distf[i] + ca + (distf[w] - distf[j]) + cb + (distf[j - 1] - distf[i + 1]) + cc + distg[w];
            int lp = 0;
            if (PD) {   // prefix(i) + run (j..w) + (i+1..j-1) + suffix(w)
                const Ld g = ld_cat(segld(j, w, false), segld(i + 1, j - 1, false));
                lp = pen(ld_close(lof[i], lmf[i], g, lig[w], lmg[w]));
            }
            TGA_TRY(dist - baseDist + wT * (tw + w3 + twg[w] - baseTw) + lp,
                    (unsigned)op * W2 + (unsigned)node[j] * W + ai);
        }
    }
}

// Intra-route candidates of a CVRP whose moved element is the customer at
// position p, with one warp (all lanes call): every delta is an O(1) edge
// formula (loads do not change inside a route), lanes take the other end j
// of the move, and each distance comes from a row segment of the
// position-ordered copy indexed by j, so a warp's loads are contiguous.
//   relocate/or-opt run i..i+k-1 after j: rem_k + c(x_j,x_i) + c(x_{i+k-1},x_{j+1}) - c(x_j,x_{j+1})
//   swap i<j (adjacent or not), 2-opt i<j (reversal of i..j).
// XS: also the swaps of runs -- x_i alone with the run x_j x_j+1 (either
// side), and the run x_i x_i+1 with a later run x_j x_j+1.
template <bool XS = false>
__device__ void intra_cvrp_position(const Dev &d, int p, int lane, int &best, unsigned &bidx) {
    if (p >= d.Wp - 1) return;
    const int ax = d.seq[TGA_IX(p, d.Wp)];
    if (ax > d.n) return;                               // a start depot is never moved
    const BRec bx = d.brec[TGA_IX(ax, d.W + 1)];
    const int r = bx.route, i = bx.idx;
    const RouteRec R = d.rrec[TGA_IX(r, d.m)];
    const int L = R.len, st = R.start;
    if (L < 2) return;
    const unsigned mask = d.op_mask;
    const unsigned W = (unsigned)d.W, W2 = W * W;
    auto nodeAt = [&](int k) { return (k <= 0 || k > L) ? 0 : d.seq[TGA_IX(st + k, d.Wp)]; };
    auto rowOf = [&](int node) { return d.pcol + (size_t)TGA_IX(node, d.n + 1) * d.ldp + TGA_IX(kColOff + st, d.ldp); };
    // distance from the prefix through element k to element k+1
    auto dfAt = [&](int k) {
        if (k > L) return R.dist;
        return d.brec[TGA_IX(k == 0 ? d.n + 1 + r : d.seq[TGA_IX(st + k, d.Wp)], d.W + 1)].distf;
    };
    const int xi = ax, xm = nodeAt(i - 1), xn = nodeAt(i + 1);
    const int *rowI = rowOf(xi), *rowP = rowOf(xm), *rowN = rowOf(xn);
    const int e_prev = dfAt(i) - dfAt(i - 1);            // c(x_{i-1}, x_i)
    const int e_next = dfAt(i + 1) - dfAt(i);            // c(x_i, x_{i+1})
    // removal gains of runs of length 1..3 starting at i
    int remk[4] = {0, 0, 0, 0};
    const int *rowW[4] = {rowI, rowI, rowI, rowI};
    for (int k = 1; k <= 3; ++k) {
        if (i + k - 1 > L) break;
        const int w = nodeAt(i + k - 1);
        rowW[k] = rowOf(w);
        const int e_w = dfAt(i + k) - dfAt(i + k - 1);  // c(x_{i+k-1}, x_{i+k})
        remk[k] = TGA_LDG(rowP + i + k) - e_prev - e_w;
    }
    for (int j = lane; j <= L; j += 32) {
        const int aj = j == 0 ? d.n + 1 + r : d.seq[TGA_IX(st + j, d.Wp)];
        const int df_j = j == 0 ? 0 : d.brec[TGA_IX(aj, d.W + 1)].distf;
        const int e_j = dfAt(j + 1) - df_j;                // c(x_j, x_{j+1})
        const int cij = TGA_LDG(rowI + j);
        for (int k = 1; k <= 3; ++k) {
            const int op = k == 1 ? 0 : k + 2;
            if (!(mask & (1u << op)) || i + k - 1 > L) continue;
            if (j >= i - 1 && j <= i + k - 1) continue;
            const int delta = remk[k] + cij + TGA_LDG(rowW[k] + j + 1) - e_j;
            TGA_TRY(delta, (unsigned)op * W2 + (unsigned)xi * W + (unsigned)aj);
        }
        if (j > i) {
            const int cpj = TGA_LDG(rowP + j), ci_j1 = TGA_LDG(rowI + j + 1);
            if (mask & 2u) {
                int delta;
                if (j == i + 1) {
                    delta = cpj + ci_j1 - e_prev - e_j;
                } else {
                    const int e_jm = df_j - dfAt(j - 1);     // c(x_{j-1}, x_j)
                    delta = cpj + TGA_LDG(rowN + j) + TGA_LDG(rowI + j - 1) + ci_j1 - e_prev - e_next - e_jm - e_j;
                }
                const unsigned xj = (unsigned)aj;
                TGA_TRY(delta, W2 + min((unsigned)xi, xj) * W + max((unsigned)xi, xj));
            }
            if (mask & 4u) {
                const int delta = cpj + ci_j1 - e_prev - e_j;
                TGA_TRY(delta, 2u * W2 + (unsigned)xi * W + (unsigned)aj);
            }
        }
        if (XS && j >= 1) {
            // e(k) = c(x_k, x_k+1), the route's edge leaving element k
            auto edge = [&](int k) { return dfAt(k + 1) - dfAt(k); };
            const unsigned xj = (unsigned)aj;
            if ((mask & 64u) && j + 1 <= L) {
                // x_i alone, the run x_j x_j+1
                int delta = kBig;
                if (j == i + 1) {            // (i-1) (i+1 i+2) (i) (i+3)
                    delta = TGA_LDG(rowP + i + 1) + TGA_LDG(rowI + i + 2) + TGA_LDG(rowI + i + 3) - e_prev - e_next -
                            edge(i + 2);
                } else if (j >= i + 2) {     // (i-1) (j j+1) (i+1..j-1) (i) (j+2)
                    delta = TGA_LDG(rowP + j) + TGA_LDG(rowN + j + 1) + TGA_LDG(rowI + j - 1) +
                            TGA_LDG(rowI + j + 2) - e_prev - e_next - edge(j - 1) - edge(j + 1);
                } else if (j == i - 2) {     // (i-3) (i) (i-2 i-1) (i+1)
                    delta = TGA_LDG(rowI + i - 3) + TGA_LDG(rowI + i - 2) + TGA_LDG(rowP + i + 1) - edge(i - 3) -
                            e_prev - e_next;
                } else if (j <= i - 3) {     // (j-1) (i) (j+2..i-1) (j j+1) (i+1)
                    delta = TGA_LDG(rowI + j - 1) + TGA_LDG(rowI + j + 2) + TGA_LDG(rowP + j) +
                            TGA_LDG(rowN + j + 1) - edge(j - 1) - edge(j + 1) - e_prev - e_next;
                }
                if (delta < kBig) TGA_TRY(delta, 6u * W2 + (unsigned)xi * W + xj);
            }
            if ((mask & 128u) && i + 1 <= L && j >= i + 2 && j + 1 <= L) {
                // the run x_i x_i+1 with the later run x_j x_j+1
                const int *rowN2 = rowOf(nodeAt(i + 2));
                const int e_i1 = edge(i + 1);        // c(x_i+1, x_i+2)
                int delta;
                if (j == i + 2) {            // (i-1) (i+2 i+3) (i i+1) (i+4)
                    delta = TGA_LDG(rowP + i + 2) + TGA_LDG(rowI + i + 3) + TGA_LDG(rowN + i + 4) - e_prev - e_i1 -
                            edge(i + 3);
                } else {                     // (i-1) (j j+1) (i+2..j-1) (i i+1) (j+2)
                    delta = TGA_LDG(rowP + j) + TGA_LDG(rowN2 + j + 1) + TGA_LDG(rowI + j - 1) +
                            TGA_LDG(rowN + j + 2) - e_prev - e_i1 - edge(j - 1) - edge(j + 1);
                }
                TGA_TRY(delta, 7u * W2 + min((unsigned)xi, xj) * W + max((unsigned)xi, xj));
            }
        }
    }
}

// Intra-route candidates of a whole CVRP route r with one warp (all lanes
// call; relocate, or-opt, swap and 2-opt, no swaps of runs).  Lane k reads
// the node of element k (0 = start depot, L+1 = end depot) and then element
// k's column of the route's (L+2) x (L+2) distance block, row by row, from
// the position-ordered copy (row x_a, columns st .. st+L+1: contiguous over
// the lanes).  The block sits in shared memory (sD, 32 x 33 ints per warp;
// sA, 32 anchors), and every candidate (i, j) is then an O(1) edge formula
// over it -- the same expressions as intra_cvrp_position:
//   relocate / or-opt run i..i+k-1 after j: c(x_i-1, x_i+k) - e(i-1) - e(i+k-1)
//       + c(x_j, x_i) + c(x_i+k-1, x_j+1) - e(j)
//   swap i < j, 2-opt i < j (reversal of i..j)
// with e(k) = c(x_k, x_k+1).  Routes of more than 30 customers take
// intra_cvrp_position for each of their customers.
constexpr int kCvrpRouteInts = 32 * 33;                 // per warp: the distance block of one route

__device__ void intra_cvrp_route(const Dev &d, int r, int lane, int *sD, int *sA, int &best, unsigned &bidx) {
    if (r >= d.m) return;
    const RouteRec R = d.rrec[TGA_IX(r, d.m)];
    const int L = R.len, st = R.start, E = L + 2;
    if (L < 2) return;
    if (E > 32) {
        for (int k = 1; k <= L; ++k) intra_cvrp_position<false>(d, st + k, lane, best, bidx);
        return;
    }
    constexpr int LD = 33;
    const int x = lane < E ? node_of(d.seq[TGA_IX(st + lane, d.Wp)], d.n) : 0;
    sA[lane] = lane == 0 ? d.n + 1 + r : x;             // anchor of element k (customers: their node)
    // eight rows per round: the loads of a round are all issued before the
    // first of them is stored
    for (int a0 = 0; a0 < E; a0 += 8) {
        int v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int xa = __shfl_sync(0xffffffffu, x, (a0 + u) & 31);
            v[u] = (a0 + u < E && lane < E)
                       ? TGA_LDG(d.pcol + (size_t)TGA_IX(xa, d.n + 1) * d.ldp + TGA_IX(kColOff + st + lane, d.ldp))
                       : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (a0 + u < E) sD[(a0 + u) * LD + lane] = v[u];
    }
    __syncwarp();
    const unsigned mask = d.op_mask;
    const unsigned W = (unsigned)d.W, W2 = W * W;
    auto D = [&](int a, int b) { return sD[a * LD + b]; };
    auto e = [&](int k) { return sD[k * LD + k + 1]; };
    const int T = L * (L + 1);
    for (int t = lane; t < T; t += 32) {
        const int i = t / (L + 1) + 1, j = t - (i - 1) * (L + 1);
        const unsigned xi = (unsigned)sA[i], aj = (unsigned)sA[j];
        const int cji = D(j, i), ej = e(j);
        for (int k = 1; k <= 3; ++k) {
            const int op = k == 1 ? 0 : k + 2;
            if (!(mask & (1u << op)) || i + k - 1 > L) continue;
            if (j >= i - 1 && j <= i + k - 1) continue;
            const int delta = D(i - 1, i + k) - e(i - 1) - e(i + k - 1) + cji + D(i + k - 1, j + 1) - ej;
            TGA_TRY(delta, (unsigned)op * W2 + xi * W + aj);
        }
        if (j > i) {
            const int cpj = D(i - 1, j), ci_j1 = D(i, j + 1);
            if (mask & 2u) {
                const int delta = j == i + 1 ? cpj + ci_j1 - e(i - 1) - ej
                                             : cpj + D(i + 1, j) + D(i, j - 1) + ci_j1 - e(i - 1) - e(i) - e(j - 1) - ej;
                TGA_TRY(delta, W2 + min(xi, aj) * W + max(xi, aj));
            }
            if (mask & 4u) TGA_TRY(cpj + ci_j1 - e(i - 1) - ej, 2u * W2 + xi * W + aj);
        }
    }
    __syncwarp();                                        // sD, sA are reused by the next route
}

// ---------------------------------------------------------------------------
// apply (tensor update of Section 5.3.5)
//
// One launch per step.  CTA 0 decodes the best key into a StepPlan,
// publishes it in Control, then rewrites the positions, the route offsets
// and the attributes of the <= 2 touched routes.  Every other CTA waits for
// the plan and permutes the changed columns of its rows of the
// position-ordered distance copy, which CTA 0 never touches.  The batched
// kernel runs the same two parts one after the other.

// Old position of the anchor that sits at index t (1-based) of the new
// route X (X is plan.A or plan.B).
__device__ __forceinline__ int new_src(const MovePlan &P, bool isA, int t) {
    const int op = P.op;
    if (P.A == P.B) {   // intra-route: index map inside route A
        int f = t;
        if (op == 0 || op == 4 || op == 5) {
            const int i = P.i, j = P.j, k = P.k;
            if (j >= i + k) {
                if (t < i) f = t;
                else if (t <= j - k) f = t + k;
                else if (t <= j) f = i + (t - (j - k + 1));
                else f = t;
            } else {    // j <= i - 2
                if (t <= j) f = t;
                else if (t <= j + k) f = i + (t - j - 1);
                else if (t <= i + k - 1) f = t - k;
                else f = t;
            }
        } else if (op == 1) {
            f = (t == P.i) ? P.j : (t == P.j ? P.i : t);
        } else if (op == 2) {
            f = (t >= P.i && t <= P.j) ? P.i + P.j - t : t;
        } else if (op >= 6) {
            // runs x (kx) before y (ky) exchange places; the middle keeps its order
            const bool af = P.i < P.j;
            const int x = af ? P.i : P.j, kx = af ? P.k : 2, y = af ? P.j : P.i, ky = af ? 2 : P.k;
            if (t < x) f = t;
            else if (t < x + ky) f = y + (t - x);
            else if (t < y + ky - kx) f = x + kx + (t - x - ky);
            else if (t < y + ky) f = x + (t - (y + ky - kx));
            else f = t;
        }
        return P.pA + f;
    }
    if (op >= 6) {      // the run of k at a and the run of 2 at b exchange routes
        if (isA) {
            if (t < P.i) return P.pA + t;
            if (t < P.i + 2) return P.pB + P.j + (t - P.i);
            return P.pA + t - 2 + P.k;
        }
        if (t < P.j) return P.pB + t;
        if (t < P.j + P.k) return P.pA + P.i + (t - P.j);
        return P.pB + t - P.k + 2;
    }
    if (op == 0 || op == 4 || op == 5) {
        if (isA) return t < P.i ? P.pA + t : P.pA + t + P.k;
        if (t <= P.j) return P.pB + t;
        if (t <= P.j + P.k) return P.pA + P.i + (t - P.j - 1);
        return P.pB + t - P.k;
    }
    if (op == 1) {
        if (isA) return t == P.i ? P.pB + P.j : P.pA + t;
        return t == P.j ? P.pA + P.i : P.pB + t;
    }
    // op 3 (2-opt*), A < B
    if (isA) return t <= P.i ? P.pA + t : P.pB + P.j + (t - P.i);
    return t <= P.j ? P.pB + t : P.pA + P.i + (t - P.j);
}

// u-th changed position of the plan.
__device__ __forceinline__ int plan_pos(const StepPlan &S, int u) {
    return u < S.n1 ? S.b1 + u : S.b2 + (u - S.n1);
}

// Old position of the anchor that lands at the changed position q.
__device__ __forceinline__ int plan_src(const StepPlan &S, int q) {
    const MovePlan &pl = S.mp;
    if (pl.A == pl.B) return new_src(pl, true, q - pl.pA);
    const bool aLo = pl.A < pl.B;
    const int plo = aLo ? pl.pA : pl.pB, phi = aLo ? pl.pB : pl.pA;
    const int nLlo = aLo ? pl.nLA : pl.nLB;
    if (q <= plo + nLlo) return new_src(pl, aLo, q - plo);
    if (q <= phi + S.dl) return q - S.dl;
    return new_src(pl, !aLo, q - (phi + S.dl));
}

// The changed positions split into the rewritten customers of the touched
// routes (positions qA0 + k for k < nA, then qB0 + k for k < nB) and the
// block of old positions [s0, s1] that moves by dl (empty when s0 > s1).
struct PlanParts {
    int qA0, nA, qB0, nB, s0, s1, dl;
};

__device__ __forceinline__ PlanParts plan_parts(const StepPlan &S) {
    const MovePlan &pl = S.mp;
    PlanParts R;
    R.dl = S.dl;
    R.s0 = 1;
    R.s1 = 0;
    if (pl.A == pl.B) {
        R.qA0 = pl.pA + 1; R.nA = pl.LA; R.qB0 = 0; R.nB = 0;
        return R;
    }
    const bool aLo = pl.A < pl.B;
    const int plo = aLo ? pl.pA : pl.pB, phi = aLo ? pl.pB : pl.pA;
    const int Llo = aLo ? pl.LA : pl.LB, nLlo = aLo ? pl.nLA : pl.nLB, nLhi = aLo ? pl.nLB : pl.nLA;
    R.qA0 = plo + 1; R.nA = nLlo;
    R.qB0 = phi + S.dl + 1; R.nB = nLhi;
    if (S.dl != 0) { R.s0 = plo + Llo + 1; R.s1 = phi; }
    return R;
}

// Index into the plan's list of changed positions of position q (q must be
// one of them).
__device__ __forceinline__ int plan_u(const StepPlan &S, int q) {
    return (q >= S.b1 && q < S.b1 + S.n1) ? q - S.b1 : S.n1 + (q - S.b2);
}

// Start-depot position of route A (isA) or B after the move.
__device__ __forceinline__ int plan_new_start(const StepPlan &S, bool isA) {
    const MovePlan &pl = S.mp;
    if (pl.A == pl.B) return pl.pA;
    const bool aLo = pl.A < pl.B;
    const int plo = aLo ? pl.pA : pl.pB, phi = aLo ? pl.pB : pl.pA;
    return (isA == aLo) ? plo : phi + S.dl;
}

__device__ __forceinline__ Seg seg_vals(int e, int l, int s, int load, int out) {
    Seg x;
    x.E = e; x.L = l; x.D = s; x.TW = 0; x.dist = 0; x.load = load; x.out = out;
    return x;
}

// Rebuild route r after a move with one warp (all lanes call), for routes
// with L + 2 <= 32 elements whose new customers are in shared memory:
// customer t (1..L) is sbuf[plan_u(S, st + t)], st = the start-depot
// position.  Produces exactly what rebuild_route does, but every global
// read is issued in one round of independent loads -- node data, the edge
// leaving each element and the bypass edges of the hoisted constants
// (x- to x+, and x- to the element after runs of 2 and 3) -- followed by
// the two concatenation scans (Section 4.3) in registers and the stores.
// Lane 0 writes the route totals (range load, dist, warp, cost) to
// tot[0..3]; the range load is the delivery total, plus the pickup total
// with pickups.
template <bool PD, bool XS = false>
__device__ void rebuild_route_warp(const Dev &d, int r, int st, int L, const int *sbuf, const StepPlan &S,
                                   int lane, int *tot) {
    const int E = L + 2;
    const bool tw = d.has_tw != 0;
    constexpr bool pd = PD;
    const int wTe = tw ? d.wT : 0;
    const unsigned mask = d.op_mask;
    const unsigned FULL = 0xffffffffu;
    const int k = lane;
    const bool valid = k < E;
    const int x = (k >= 1 && k <= L) ? sbuf[plan_u(S, st + k)] : 0;   // node (depots are 0)
    const int xn = __shfl_down_sync(FULL, x, 1), xm = __shfl_up_sync(FULL, x, 1);
    const int x2 = __shfl_down_sync(FULL, x, 2), x3 = __shfl_down_sync(FULL, x, 3);
    // ---- one round of loads
    const int out = (valid && k + 1 < E) ? dmat(d, x, k + 1 <= L ? xn : 0) : 0;
    const int dem = __ldg(d.demand + x);
    const int ne = tw ? __ldg(d.early + x) : 0, nl = tw ? __ldg(d.late + x) : 0;
    const int ns = tw ? __ldg(d.service + x) : 0;
    const bool cust = k >= 1 && k <= L;
    const int cmn = cust ? dmat(d, xm, k + 1 <= L ? xn : 0) : 0;
    const int c2 = (cust && k + 1 <= L) ? dmat(d, xm, k + 2 <= L ? x2 : 0) : 0;
    const int c3 = (cust && k + 2 <= L) ? dmat(d, xm, k + 3 <= L ? x3 : 0) : 0;
    // ---- forward scan: prefix through element k
    const Seg node = seg_vals(ne, nl, ns, dem, out);
    Seg f = node;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        Seg o = shfl_seg_up(f, off);
        if (lane >= off) f = seg_cat(o, f);
    }
    // ---- backward scan: elements k .. L+1
    Seg g = node;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        Seg o = shfl_seg_down(g, off);
        if (lane + off < E) g = seg_cat(g, o);
    }
    // pickups: the same two scans of the loads (Section 4.3.2)
    Ld ndl{0, 0, 0}, fl{0, 0, 0}, gl{0, 0, 0};
    if (pd) {
        ndl = ld_node(d, x);
        fl = ndl;
        gl = ndl;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const Ld o = shfl_ld_up(fl, off);
            if (lane >= off) fl = ld_cat(o, fl);
            const Ld p = shfl_ld_down(gl, off);
            if (lane + off < E) gl = ld_cat(gl, p);
        }
    }
    // route totals: the prefix of the end depot
    const int Rload = __shfl_sync(FULL, f.load, E - 1);
    const int Rdist = __shfl_sync(FULL, f.dist, E - 1);
    const int Rtw = tw ? __shfl_sync(FULL, f.TW, E - 1) : 0;
    const int Rlo = pd ? __shfl_sync(FULL, fl.o, E - 1) : 0;
    const int Rlm = pd ? __shfl_sync(FULL, fl.m, E - 1) : Rload;
    const int Rcost = L == 0 ? 0 : Rdist + d.wL * max(Rlm - d.Q, 0) + wTe * Rtw;
    // own record: prefix through x, suffix after x (= backward scan at k+1)
    const int tau = tw ? f.E + f.D - f.TW : 0, twf = tw ? f.TW : 0;
    const int gL = __shfl_down_sync(FULL, g.L, 1), gTW = __shfl_down_sync(FULL, g.TW, 1);
    const int gdist = __shfl_down_sync(FULL, g.dist, 1), gload = __shfl_down_sync(FULL, g.load, 1);
    const int Lg = tw ? gL : 0, twg = tw ? gTW : 0;
    // predecessor's prefix, and the suffixes after the last element of the
    // runs x..x+1 and x..x+2 (the records of elements k+1 and k+2)
    const int ptau = __shfl_up_sync(FULL, tau, 1), ptwf = __shfl_up_sync(FULL, twf, 1);
    const int pdist = __shfl_up_sync(FULL, f.dist, 1);
    const int w2L = __shfl_down_sync(FULL, Lg, 1), w2tw = __shfl_down_sync(FULL, twg, 1);
    const int w2dist = __shfl_down_sync(FULL, gdist, 1);
    const int w3L = __shfl_down_sync(FULL, Lg, 2), w3tw = __shfl_down_sync(FULL, twg, 2);
    const int w3dist = __shfl_down_sync(FULL, gdist, 2);
    // the runs x..x+1 and x..x+2
    const Seg n1 = shfl_seg_down(node, 1), n2 = shfl_seg_down(node, 2);
    const Seg run2 = seg_cat(node, n1), run3 = seg_cat(run2, n2);
    const int dnext = XS ? __shfl_down_sync(FULL, dem, 1) : 0;       // demand of x+
    // pickups: suffix loads after x, after x+1 and after x+2; prefix loads
    // through x-; the loads of the runs
    int glI = 0, glM = 0, w2I = 0, w2M = 0, w3I = 0, w3M = 0, plo = 0, plm = 0;
    Ld r2l{0, 0, 0}, r3l{0, 0, 0};
    if (pd) {
        glI = __shfl_down_sync(FULL, gl.i, 1); glM = __shfl_down_sync(FULL, gl.m, 1);
        w2I = __shfl_down_sync(FULL, glI, 1); w2M = __shfl_down_sync(FULL, glM, 1);
        w3I = __shfl_down_sync(FULL, glI, 2); w3M = __shfl_down_sync(FULL, glM, 2);
        plo = __shfl_up_sync(FULL, fl.o, 1); plm = __shfl_up_sync(FULL, fl.m, 1);
        const Ld m1 = shfl_ld_down(ndl, 1), m2 = shfl_ld_down(ndl, 2);
        r2l = ld_cat(ndl, m1);
        r3l = ld_cat(r2l, m2);
    }
    if (k <= L) {
        const int a = k == 0 ? d.n + 1 + r : x;
        int4 *bp = reinterpret_cast<int4 *>(d.brec + TGA_IX(a, d.W + 1));
        bp[0] = make_int4(x, r, k, L);
        bp[1] = make_int4(tau, twf, f.dist, f.load);
        bp[2] = make_int4(Lg, twg, gdist, gload);
        bp[3] = make_int4(Rcost, fl.o, fl.m, glM);
        const int Fc = f.dist + wTe * twf - Rcost;
        const int Gc = gdist + wTe * twg;
        int rem1 = kBig, K2 = kBig, LQd = 0, tauP = 0;
        int C2 = kBig, ld2 = 0, E2 = 0, L2 = 0, Dm2 = 0;
        int C3 = kBig, ld3 = 0, E3 = 0, L3 = 0, Dm3 = 0;
        if (k >= 1) {
            const int twr = tw ? ptwf + twg + max(ptau + cmn - Lg, 0) : 0;
            const int lrem = pd ? max(plm + glI, plo + glM) : Rload - dem;
            const int c1 = pdist + cmn + gdist + d.wL * max(lrem - d.Q, 0) + wTe * twr;
            rem1 = c1 - Rcost + ((mask & 1u) ? 0 : kBig);
            K2 = pdist + gdist + wTe * (ptwf + twg) - Rcost + ((mask & 2u) ? 0 : kBig);
            LQd = Rload - dem - d.Q;
            tauP = ptau;
            if (k + 1 <= L && (mask & 16u)) {
                const int twk = tw ? ptwf + w2tw + max(ptau + c2 - w2L, 0) : 0;
                const int lk = pd ? max(plm + w2I, plo + w2M) : Rload - run2.load;
                const int ck = pdist + c2 + w2dist + d.wL * max(lk - d.Q, 0) + wTe * twk - Rcost;
                C2 = ck + run2.dist + wTe * (tw ? run2.TW : 0);
                ld2 = run2.load;
                if (tw) { E2 = run2.E; L2 = run2.L; Dm2 = run2.D - run2.TW; }
            }
            if (k + 2 <= L && (mask & 32u)) {
                const int twk = tw ? ptwf + w3tw + max(ptau + c3 - w3L, 0) : 0;
                const int lk = pd ? max(plm + w3I, plo + w3M) : Rload - run3.load;
                const int ck = pdist + c3 + w3dist + d.wL * max(lk - d.Q, 0) + wTe * twk - Rcost;
                C3 = ck + run3.dist + wTe * (tw ? run3.TW : 0);
                ld3 = run3.load;
                if (tw) { E3 = run3.E; L3 = run3.L; Dm3 = run3.D - run3.TW; }
            }
        }
        int4 *ep = reinterpret_cast<int4 *>(d.erec + TGA_IX(a, d.W + 1));
        ep[0] = make_int4(r, dem, rem1, Fc + Gc);
        ep[1] = make_int4(Rload - d.Q, K2, LQd, Fc + ((mask & 8u) ? 0 : kBig));
        ep[2] = make_int4(Gc, f.load, gload - d.Q, a);
        ep[3] = make_int4(C2, ld2, C3, ld3);
        ep[4] = make_int4(ne, nl, ns, tau);
        ep[5] = make_int4(Lg, tauP, E2, L2);
        ep[6] = make_int4(Dm2, E3, L3, Dm3);
        ep[7] = make_int4(x, k, k + 1 <= L ? xn : 0, k + 2 <= L ? x2 : 0);
        if (XS) {
            d.xrec[TGA_IX(a, d.W + 1)] = k == 0 ? xrec_none()
                               : make_xrec(wTe, Rcost, Rload, d.Q, pdist, ptwf, ptau, gdist, twg, Lg, k + 1 <= L,
                                           w2dist, w2tw, w2L, run2, dnext, ne, nl, ns, dem);
        }
        if (pd) {
            const int Q = d.Q;
            const int pk = ndl.o;
            int4 *pp = reinterpret_cast<int4 *>(d.prec + TGA_IX(a, d.W + 1));
            pp[0] = make_int4(fl.m + glI - Q, fl.o + glI - Q, fl.o + glM - Q, pk);
            pp[1] = k >= 1 ? make_int4(plm + glI - Q, plo + glI - Q, plo + glM - Q, max(dem, pk))
                           : make_int4(0, 0, 0, max(dem, pk));
            pp[2] = make_int4(fl.m - Q, fl.o - Q, glI, glM);
            pp[3] = make_int4(C2 < kBig ? r2l.o : 0, C2 < kBig ? r2l.m : 0, C3 < kBig ? r3l.o : 0,
                              C3 < kBig ? r3l.m : 0);
        }
    }
    if (lane == 0) {
        RouteRec *R = d.rrec + TGA_IX(r, d.m);
        R->load = Rload;
        if (pd) { R->lo = Rlo; R->lm = Rlm; }
        R->dist = Rdist;
        R->tw = Rtw;
        R->cost = Rcost;
        tot[0] = pd ? Rload + Rlo : Rload; tot[1] = Rdist; tot[2] = Rtw; tot[3] = Rcost;
    }
}

// Decode the step's move -- the evaluation's packed best key, or *ext --
// into S (one thread).  S.act = 0 when there is nothing to apply: a local
// optimum, a context that is done, or an invalid move (status set).
__device__ void decode_plan(const Dev &d, const tga_move *ext, StepPlan &S) {
    Control *C = d.ctl;
    S.act = 0;
    // the stop flag, the status and the best key in one round trip (the
    // loads are issued together, before any of them is tested)
    const int done = *(volatile int *)&C->done;
    const int status = *(volatile int *)&C->status;
    const unsigned long long best = *(volatile unsigned long long *)&C->best_key;
    if (done && !ext) return;
    if (!ext && status != 0) {                 // an error found during the last step ends the descent
        C->done = 1;
        return;
    }
    const unsigned long long key = ext ? (ext->valid ? pack_key(ext->delta, ext->move_index) : kNoKey) : best;
    const bool improving = key != kNoKey && key_delta(key) < 0;
    const unsigned idx = (unsigned)(key & 0xffffffffu);
    const unsigned W = (unsigned)d.W, W2 = W * W;
    MovePlan pl;
    pl.op = (int)(idx / W2);
    pl.a = (int)((idx % W2) / W);
    pl.b = (int)(idx % W);
    pl.delta = key_delta(key);
    bool ok = improving && pl.op < 8 && ((d.op_mask >> pl.op) & 1u) && pl.a >= 1 && pl.b >= 1 &&
              pl.a < d.W && pl.b < d.W;
    int costA = 0, costB = 0;
    BRec ba{}, bb{};
    int qa = 0, qb = 0;
    if (ok) {
        // one round trip: the anchors' records carry route, index, route
        // length and cost; the start depot sits idx positions before the anchor
        ba = d.brec[TGA_IX(pl.a, d.W + 1)]; bb = d.brec[TGA_IX(pl.b, d.W + 1)];
        qa = d.pos_of[TGA_IX(pl.a, d.W + 1)]; qb = d.pos_of[TGA_IX(pl.b, d.W + 1)];
    }
    // the evaluation's bookkeeping, while the records are in flight
    if (!ext) {
        if (d.log && C->evals < d.log_cap) d.log[C->evals] = key;
        count_evaluation(d, C);
    }
    C->best_key = kNoKey;
    if (!improving) {
        C->done = 1;
        C->local_opt = 1;
        return;
    }
    if (ok) {
        pl.A = ba.route; pl.B = bb.route; pl.i = ba.idx; pl.j = bb.idx;
        pl.LA = ba.rlen; pl.LB = bb.rlen;
        pl.pA = qa - ba.idx; pl.pB = qb - bb.idx;
        costA = ba.rcost; costB = bb.rcost;
        ok = pl.A >= 0 && pl.B >= 0;
    }
    if (ok) {
        const int op = pl.op;
        pl.k = 1;
        if (op == 0 || op == 4 || op == 5) {
            pl.k = op == 0 ? 1 : op - 2;
            ok = pl.a <= d.n && pl.i + pl.k - 1 <= pl.LA &&
                 !(pl.A == pl.B && pl.j >= pl.i - 1 && pl.j <= pl.i + pl.k - 1);
            pl.nLA = pl.A == pl.B ? pl.LA : pl.LA - pl.k;
            pl.nLB = pl.A == pl.B ? pl.LB : pl.LB + pl.k;
        } else if (op == 1) {
            ok = pl.a < pl.b && pl.b <= d.n;
            pl.nLA = pl.LA; pl.nLB = pl.LB;
            if (ok && pl.A == pl.B && pl.i > pl.j) { int t = pl.i; pl.i = pl.j; pl.j = t; }
        } else if (op == 2) {
            ok = pl.a <= d.n && pl.b <= d.n && pl.A == pl.B && pl.i < pl.j;
            pl.nLA = pl.LA; pl.nLB = pl.LB;
        } else if (op >= 6) {
            // a run of k (1 or 2) at a and a run of 2 at b, disjoint
            pl.k = op == 6 ? 1 : 2;
            ok = pl.a <= d.n && pl.b <= d.n && (op == 6 || pl.a < pl.b) && pl.i + pl.k - 1 <= pl.LA &&
                 pl.j + 1 <= pl.LB && (pl.A != pl.B || pl.i + pl.k <= pl.j || pl.j + 2 <= pl.i);
            pl.nLA = pl.A == pl.B ? pl.LA : pl.LA - pl.k + 2;
            pl.nLB = pl.A == pl.B ? pl.LB : pl.LB - 2 + pl.k;
        } else {
            ok = pl.A < pl.B;
            pl.nLA = pl.i + pl.LB - pl.j;
            pl.nLB = pl.j + pl.LA - pl.i;
        }
    }
    if (!ok) {
        set_status(C, TGA_ERR_INVALID);
        C->done = 1;
        return;
    }
    S.mp = pl;
    S.act = 1;
    C->last_op = pl.op; C->last_a = pl.a; C->last_b = pl.b; C->last_delta = pl.delta;
    S.oldcost = (long long)costA + (pl.A != pl.B ? costB : 0);
    S.oldLA = pl.LA; S.oldLB = pl.LB;
    if (pl.A == pl.B) {
        S.lo = pl.A; S.hi = pl.A; S.dl = 0;
        S.b1 = pl.pA + 1; S.n1 = pl.LA; S.b2 = 0; S.n2 = 0;
    } else {
        const bool aLo = pl.A < pl.B;
        const int lo = aLo ? pl.A : pl.B, hi = aLo ? pl.B : pl.A;
        const int Llo = aLo ? pl.LA : pl.LB, nLlo = aLo ? pl.nLA : pl.nLB;
        const int plo = aLo ? pl.pA : pl.pB, phi = aLo ? pl.pB : pl.pA;
        const int Lhi = aLo ? pl.LB : pl.LA;
        S.lo = lo; S.hi = hi;
        S.dl = nLlo - Llo;
        if (S.dl != 0) {
            S.b1 = plo + 1; S.n1 = phi + Lhi - plo; S.b2 = 0; S.n2 = 0;
        } else {
            S.b1 = plo + 1; S.n1 = Llo; S.b2 = phi + 1; S.n2 = Lhi;
        }
    }
}

// Rewrite positions, route offsets and the attributes of the touched routes
// for plan S with the whole block (at least 3 warps); sbuf holds n1 + n2
// ints.  Warps 0 and 1 rebuild routes A and B -- from the new customers in
// sbuf when a route fits one warp, else with the chunked scans -- while the
// other warps find the longest route and heaviest load of the rest and one
// thread prefetches the counters.  Thread 0 then updates cost and counters
// and ends the step (done flag, graph condition); it returns 1 when the
// descent ends with this step (other threads return 0).  ext: the move came
// from the caller, whose delta is not checked against the rebuilt routes.
template <bool PD, bool XS = false>
__device__ int apply_plan_block(const Dev &d, const StepPlan &S, int *sbuf, bool ext,
                                cudaGraphConditionalHandle cond, int use_cond) {
    Control *C = d.ctl;
    int stop = 0;                             // thread 0: the descent ends with this step
    __shared__ int s_maxL, s_maxLoad;
    __shared__ int s_tot[2][4];
    __shared__ int s_fast[2];
    __shared__ long long s_cf[6];             // cost, steps, sumL2, sumLm1, sumLm2, step_limit
    __shared__ int s_ci[6];                   // status, maxc, maxl, maxe, maxs, maxd
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid == 0) { s_maxL = 0; s_maxLoad = 0; }
    if (S.act) {
        const MovePlan pl = S.mp;
        const int tot = S.n1 + S.n2;
        // the anchor every changed position takes, all read before any write
        // (eight per thread and round, their loads issued together)
        for (int u0 = tid; u0 < tot; u0 += 8 * nthr) {
            int v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int u = u0 + k * nthr;
                v[k] = u < tot ? d.seq[TGA_IX(plan_src(S, plan_pos(S, u)), d.Wp)] : 0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (u0 + k * nthr < tot) sbuf[u0 + k * nthr] = v[k];
        }
        __syncthreads();
        for (int u = tid; u < tot; u += nthr) {
            const int q = plan_pos(S, u), a = sbuf[u];
            d.seq[TGA_IX(q, d.Wp)] = a;
            d.pos_of[TGA_IX(a, d.W + 1)] = q;
        }
        if (S.dl != 0) {
            for (int r0 = S.lo + 1 + tid; r0 <= S.hi; r0 += 8 * nthr) {
                int v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int r = r0 + k * nthr;
                    v[k] = r <= S.hi ? d.rrec[TGA_IX(r, d.m)].start : 0;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (r0 + k * nthr <= S.hi) d.rrec[TGA_IX(r0 + k * nthr, d.m)].start = v[k] + S.dl;
            }
        }
        if (tid == 0) {
            d.rrec[TGA_IX(pl.A, d.m)].len = pl.nLA;
            if (pl.B != pl.A) d.rrec[TGA_IX(pl.B, d.m)].len = pl.nLB;
        }
        __syncthreads();
        const int warp = tid >> 5, lane = tid & 31;
        if (warp <= 1) {
            const bool isA = warp == 0;
            if (isA || pl.B != pl.A) {
                const int r = isA ? pl.A : pl.B, L = isA ? pl.nLA : pl.nLB;
                const bool fast = L + 2 <= 32;
                if (fast) rebuild_route_warp<PD, XS>(d, r, plan_new_start(S, isA), L, sbuf, S, lane, s_tot[warp]);
                else rebuild_route<PD, XS>(d, r, lane);
                if (lane == 0) s_fast[warp] = fast;
            }
        } else {
            if (tid == 64) {
                s_cf[0] = C->cost; s_cf[1] = C->steps; s_cf[2] = C->sumL2;
                s_cf[3] = C->sumLm1; s_cf[4] = C->sumLm2; s_cf[5] = C->step_limit;
                s_ci[0] = C->status; s_ci[1] = C->maxc; s_ci[2] = C->maxl;
                s_ci[3] = C->maxe; s_ci[4] = C->maxs; s_ci[5] = C->maxd;
            }
            // meanwhile: longest route and heaviest load of the other routes
            // (eight routes per thread and round, their loads issued together)
            int mL = 0, mLoad = 0;
            const int rstep = nthr - 64;
            for (int r0 = tid - 64; r0 < d.m; r0 += 8 * rstep) {
                int len[8], ld[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int r = r0 + u * rstep;
                    const bool in = r < d.m && r != pl.A && r != pl.B;
                    const RouteRec *Rr = d.rrec + TGA_IX(in ? r : 0, d.m);
                    len[u] = in ? Rr->len : 0;
                    ld[u] = in ? (PD ? Rr->load + Rr->lo : Rr->load) : 0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    mL = max(mL, len[u]);
                    mLoad = max(mLoad, ld[u]);
                }
            }
            mL = __reduce_max_sync(0xffffffffu, mL);
            mLoad = __reduce_max_sync(0xffffffffu, mLoad);
            if (lane == 0) { atomicMax(&s_maxL, mL); atomicMax(&s_maxLoad, mLoad); }
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (S.act) {
            const MovePlan &pl = S.mp;
            const bool two = pl.B != pl.A;
            int costA, loadA, costB = 0, loadB = 0;
            // range load: the delivery total, plus the pickup total with pickups
            auto rload = [&](int r) { return d.rrec[TGA_IX(r, d.m)].load + (PD ? d.rrec[TGA_IX(r, d.m)].lo : 0); };
            if (s_fast[0]) { costA = s_tot[0][3]; loadA = s_tot[0][0]; }
            else { costA = d.rrec[TGA_IX(pl.A, d.m)].cost; loadA = rload(pl.A); }
            if (two) {
                if (s_fast[1]) { costB = s_tot[1][3]; loadB = s_tot[1][0]; }
                else { costB = d.rrec[TGA_IX(pl.B, d.m)].cost; loadB = rload(pl.B); }
            }
            const long long newcost = (long long)costA + costB;
            const long long dact = newcost - S.oldcost;
            int status = s_ci[0];
            if (!ext && dact != pl.delta) { set_status(C, TGA_ERR_CHECK); status = TGA_ERR_CHECK; }
            const long long cost = s_cf[0] + dact, steps = s_cf[1] + 1;
            C->cost = cost;
            C->steps = steps;
            if (two) {
                auto sq = [](long long x) { return x * x; };
                const int oA = S.oldLA, oB = S.oldLB;
                const long long l2 = s_cf[2] + sq(pl.nLA) + sq(pl.nLB) - sq(oA) - sq(oB);
                const long long l1 = s_cf[3] + max(pl.nLA - 1, 0) + max(pl.nLB - 1, 0) - max(oA - 1, 0) -
                                     max(oB - 1, 0);
                const long long lm2 = s_cf[4] + max(pl.nLA - 2, 0) + max(pl.nLB - 2, 0) - max(oA - 2, 0) -
                                      max(oB - 2, 0);
                C->sumL2 = l2; C->sumLm1 = l1; C->sumLm2 = lm2;
                C->cand_per_eval = candidate_count(d.n, d.m, d.op_mask, l2, l1, lm2);
                auto sqp = [&](int x) { return x > 0 ? (long long)x * x : 0LL; };
                C->sumLm1sq += sqp(pl.nLA - 1) + sqp(pl.nLB - 1) - sqp(oA - 1) - sqp(oB - 1);
                C->sumLm2sq += sqp(pl.nLA - 2) + sqp(pl.nLB - 2) - sqp(oA - 2) - sqp(oB - 2);
            }
            const int maxL = max(s_maxL, max(pl.nLA, two ? pl.nLB : 0));
            const int maxLoad = max(s_maxLoad, max(loadA, two ? loadB : 0));
            C->maxL = maxL;
            C->maxLoad = maxLoad;
            if (!range_ok_vals(d, maxL, maxLoad, s_ci[1], s_ci[2], s_ci[3], s_ci[4], s_ci[5])) {
                set_status(C, TGA_ERR_RANGE);
                status = TGA_ERR_RANGE;
            }
            stop = status != 0 || steps >= s_cf[5];
            if (stop) C->done = 1;
            if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
        } else {
            // a stop (error or step limit) also ends host-launched descents
            if (C->status != 0 || C->steps >= C->step_limit) C->done = 1;
            stop = *(volatile int *)&C->done != 0 || C->steps >= C->step_limit;
            if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
        }
    }
    return stop;
}

// row[t + dl] = row[t] for t in [s0, s1], one warp: passes of 8 x 32 values
// whose loads all complete before their stores, walking against the shift
// so that no pass reads a value an earlier pass wrote.
__device__ __forceinline__ void shift_row_warp(int *row, int s0, int s1, int dl, int lane) {
    constexpr int P = 8;
    if (dl > 0) {
        for (int hi = s1; hi >= s0; hi -= 32 * P) {
            int v[P];
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int t = hi - 32 * k - lane;
                v[k] = t >= s0 ? row[t] : 0;
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int t = hi - 32 * k - lane;
                if (t >= s0) row[t + dl] = v[k];
            }
            __syncwarp();
        }
    } else {
        for (int lo = s0; lo <= s1; lo += 32 * P) {
            int v[P];
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int t = lo + 32 * k + lane;
                v[k] = t <= s1 ? row[t] : 0;
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int t = lo + 32 * k + lane;
                if (t <= s1) row[t + dl] = v[k];
            }
            __syncwarp();
        }
    }
}

// The same with the whole block (passes of 4 x blockDim values).
__device__ void shift_row_block(int *row, int s0, int s1, int dl) {
    constexpr int P = 4;
    const int nthr = blockDim.x, tid = threadIdx.x, step = P * nthr;
    if (dl > 0) {
        for (int hi = s1; hi >= s0; hi -= step) {
            int v[P];
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int t = hi - nthr * k - tid;
                v[k] = t >= s0 ? row[t] : 0;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int t = hi - nthr * k - tid;
                if (t >= s0) row[t + dl] = v[k];
            }
            __syncthreads();
        }
    } else {
        for (int lo = s0; lo <= s1; lo += step) {
            int v[P];
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int t = lo + nthr * k + tid;
                v[k] = t <= s1 ? row[t] : 0;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int t = lo + nthr * k + tid;
                if (t <= s1) row[t + dl] = v[k];
            }
            __syncthreads();
        }
    }
}

constexpr int kBandListMax = 1024;   // rewritten route elements listed in shared memory
constexpr int kBandWarpBuf = 256;    // per-warp values of one row (route elements)

// Shared memory (ints) the column permutation needs with nw warps.
__host__ __device__ inline int band_smem_ints(int Wp, int nw) {
    const int a = 2 * kBandListMax + nw * kBandWarpBuf;
    return Wp > a ? Wp : a;
}

// Permute the columns of the position-ordered copy for plan S, rows
// [row_lo, row_hi) shared among ncta CTAs of which this is number cta: a
// warp per row while the rewritten route elements fit the per-warp buffer,
// else a block per row.  Per row, the sources of the rewritten elements are
// read first, then the block between the two routes shifts, then the
// elements are written.  smem: band_smem_ints(Wp, warps) ints.
__device__ void band_plan_rows(const Dev &d, const StepPlan &S, int *smem, int row_lo, int row_hi, int cta,
                               int ncta) {
    if (!S.act) return;
    if (row_hi > d.n + 1) row_hi = d.n + 1;
    const PlanParts P = plan_parts(S);
    const int nL = P.nA + P.nB;
    const bool shift = P.s0 <= P.s1;
    const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    auto qk = [&](int k) { return k < P.nA ? P.qA0 + k : P.qB0 + (k - P.nA); };
    __shared__ int s_cnt;
    if (nL <= kBandListMax) {
        int *sq = smem, *ss = smem + kBandListMax;
        if (tid == 0) s_cnt = 0;
        __syncthreads();
        for (int k = tid; k < nL; k += nthr) {
            const int q = qk(k), src = plan_src(S, q);
            if (src != q) {
                const int e = atomicAdd(&s_cnt, 1);
                sq[e] = q;
                ss[e] = src;
            }
        }
        __syncthreads();
        const int K = s_cnt;
        if (K <= 32 && (!shift || P.s1 - P.s0 < 256)) {
            // one pass per row: a warp issues the loads of two rows (the
            // rewritten elements' sources and the block between the routes)
            // before any store, then shifts, then writes the elements
            const int src = lane < K ? ss[lane] : 0, dst = lane < K ? sq[lane] : 0;
            const int stride = ncta * nw;
            for (int x0 = row_lo + cta * nw + warp; x0 < row_hi; x0 += 2 * stride) {
                int g[2], v[2][8];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int x = x0 + r * stride;
                    const bool ok = x < row_hi;
                    const int *row = d.pcol + (size_t)TGA_IX(ok ? x : 0, d.n + 1) * d.ldp + kColOff;
                    g[r] = (ok && lane < K) ? row[TGA_IX(src, d.ldp - kColOff)] : 0;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int t = P.s0 + 32 * k + lane;
                        v[r][k] = (ok && shift && t <= P.s1) ? row[TGA_IX(t, d.ldp - kColOff)] : 0;
                    }
                }
                __syncwarp();
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int x = x0 + r * stride;
                    if (x >= row_hi) continue;
                    int *row = d.pcol + (size_t)TGA_IX(x, d.n + 1) * d.ldp + kColOff;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int t = P.s0 + 32 * k + lane;
                        if (shift && t <= P.s1) row[TGA_IX(t + P.dl, d.ldp - kColOff)] = v[r][k];
                    }
                }
                __syncwarp();
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int x = x0 + r * stride;
                    if (x < row_hi && lane < K) d.pcol[(size_t)TGA_IX(x, d.n + 1) * d.ldp + kColOff + TGA_IX(dst, d.ldp - kColOff)] = g[r];
                }
                __syncwarp();
            }
            return;
        }
        if (K <= kBandWarpBuf) {
            int *wb = smem + 2 * kBandListMax + warp * kBandWarpBuf;
            for (int x = row_lo + cta * nw + warp; x < row_hi; x += ncta * nw) {
                int *row = d.pcol + (size_t)TGA_IX(x, d.n + 1) * d.ldp + kColOff;
                for (int e = lane; e < K; e += 32) wb[e] = row[ss[e]];
                __syncwarp();
                if (shift) shift_row_warp(row, P.s0, P.s1, P.dl, lane);
                for (int e = lane; e < K; e += 32) row[sq[e]] = wb[e];
                __syncwarp();
            }
            return;
        }
        __syncthreads();                 // the lists are overwritten below
    }
    // long routes: a block per row, sources recomputed per element
    int *vb = smem;
    for (int x = row_lo + cta; x < row_hi; x += ncta) {
        int *row = d.pcol + (size_t)TGA_IX(x, d.n + 1) * d.ldp + kColOff;
        for (int k = tid; k < nL; k += nthr) vb[k] = row[plan_src(S, qk(k))];
        __syncthreads();
        if (shift) shift_row_block(row, P.s0, P.s1, P.dl);
        for (int k = tid; k < nL; k += nthr) row[qk(k)] = vb[k];
        __syncthreads();
    }
}

// Write the caller's giant tour and route offsets from the device state
// (positions, per-anchor routes, route start positions); grid-stride.
__device__ void sync_solution_range(const Dev &d, long long t0, long long stride) {
    if (*(volatile int *)&d.ctl->status != 0) return;     // an error leaves the caller's solution as it was
    for (long long q = t0; q < d.Wp - 1; q += stride) {
        const int a = d.seq[TGA_IX(q, d.Wp)];
        if (a >= 1 && a <= d.n) d.tour[TGA_IX(q - d.brec[TGA_IX(a, d.W + 1)].route - 1, d.n)] = a;
    }
    for (long long r = t0; r <= d.m; r += stride)
        d.route_start[TGA_IX(r, d.m + 1)] = r < d.m ? d.rrec[TGA_IX(r, d.m)].start - (int)r : d.n;
}

__device__ __forceinline__ long long now_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (one thread) until *flag != 0, at most limit_ns; false on timeout.
__device__ bool wait_flag(const int *flag, long long limit_ns) {
    const long long t0 = now_ns();
    while (*(const volatile int *)flag == 0) {
        if (now_ns() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// Copy the published plan into shared memory (whole block; L1 bypassed).
__device__ void load_plan(const Control *C, StepPlan *dst) {
    const volatile int *src = reinterpret_cast<const volatile int *>(&C->plan);
    int *o = reinterpret_cast<int *>(dst);
    for (int t = threadIdx.x; t < (int)(sizeof(StepPlan) / sizeof(int)); t += blockDim.x) o[t] = src[t];
}

// Last-block-done tail of a descent step's evaluation (thread 0 of every CTA
// of the step's evaluation launches, after its key is folded in): the CTA
// that finishes last decodes the best key into the step's plan, read by the
// apply launch that follows on the stream.  The count re-arms itself.
__device__ void eval_tail(const Dev &d, int total) {
    Control *C = d.ctl;
    // release: this CTA's key is folded in; acquire: so are all the others'
    if (atom_add_acq_rel(&C->eval_done, 1) != total - 1) return;
    C->eval_done = 0;
    StepPlan P;
    decode_plan(d, nullptr, P);
    C->plan = P;
    C->plan_ready = 1;
}


}  // namespace
}  // namespace tga
