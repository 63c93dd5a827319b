// Single-instance descent in one persistent launch.
//
// The graph path runs every local-search step as separate kernel launches
// (inter-route and intra-route evaluation, then apply).  For instances of a
// few thousand customers or fewer, a step holds only microseconds of
// arithmetic, so the gaps between dependent launches and the ramp of each
// grid are a large share of the step.  Here one cooperative launch keeps
// every CTA resident for the whole descent (Appendix algorithm "Feasible and
// infeasible search": evaluate, pick the best improving move, apply, repeat):
//
//   evaluation   every CTA takes the inter-route tiles and intra-route items
//                {blockIdx, blockIdx + G, ...} (Section 5.3.1-5.3.3, the
//                same device functions as the per-step kernels) and folds
//                them into the packed best key (Section 5.3.4, Eq. "min_obj");
//   decode       the last CTA to finish decodes the key into the step's plan
//                and publishes it; every other CTA waits for the publication
//                (this wait is the step's first synchronisation point);
//   update       the decoding CTA applies the move (Section 5.3.5, rewriting
//                positions and the <= 2 touched routes); the other CTAs
//                permute the columns of the position-ordered distance copy;
//   barrier      then the next step, until the move is not improving or the
//                step limit is reached.  The caller's giant tour is written
//                back by the next launch on the stream (k_sync_solution),
//                once every CTA has stopped, and only if no wait ran out.
//
// A cooperative launch guarantees that all CTAs are resident at once, so
// the grid barriers cannot deadlock; each wait still has a time limit after
// which the descent stops with TGA_ERR_TIMEOUT.  Compiled like the batched
// kernel: plain loads with L1 caching of global data disabled, because
// another SM rewrites the search state within the launch.
#define TGA_LDG(p) (*(p))
#include "tga_device.cuh"
#undef TGA_FILE_ID
#define TGA_FILE_ID 4

namespace tga {

namespace {

// Grid barrier: each CTA adds one to an arrival count that only grows
// within the launch; the k-th barrier (k = 1, 2, ...) is passed when the
// count reaches k * G.  The CTA that ends the descent adds kStopFlag beside
// its arrival, so every CTA learns of the stop from the load that passes the
// barrier (no further read of the stop flag).  One thread per CTA waits, at
// most limit_ns.  Returns 0 on timeout, 1 when passed, 2 when passed and the
// descent ends.
constexpr unsigned long long kStopFlag = 1ull << 40;

__device__ int grid_barrier(unsigned long long *count, unsigned long long target, bool stop, long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        red_add_release(count, stop ? kStopFlag + 1 : 1ull);   // publishes the block's writes
        int ok = 1;
        unsigned long long v = ld_acquire(count);
        if ((v & (kStopFlag - 1)) < target) {
            const long long t0 = now_ns();
            while (((v = ld_acquire(count)) & (kStopFlag - 1)) < target) {
                if (now_ns() - t0 > limit_ns) { ok = 0; break; }
            }
        }
        s_ok = ok ? (v >= kStopFlag ? 2 : 1) : 0;
    }
    __syncthreads();
    return s_ok;
}

// Wait (one thread) until *seq == want, at most limit_ns (acquire).
__device__ bool wait_seq(const int *seq, int want, long long limit_ns) {
    if (ld_acquire(seq) != want) {
        const long long t0 = now_ns();
        while (ld_acquire(seq) != want)
            if (now_ns() - t0 > limit_ns) return false;
    }
    return true;
}

}  // namespace

// ntiles inter-route tiles (TR rows x 32 * warps / RS columns each) and
// nintra intra-route items: one route per item with time windows, else
// blockDim/32 routes per item (one warp each, intra_cvrp_route) or, for long
// CVRP routes, blockDim/32 moved customers per item (intra_cvrp_position).
// STRIP (RS = 0): strip mode -- after the intra-route items every CTA walks its
// contiguous share of the ntiles tiles of the strip-major order (TR rows x
// 32 * warps columns, strip_walk), as the per-step strip kernel does, so a
// large instance runs its whole descent in this one launch too.
// PD: pickups (with time windows).
template <bool TW, bool OR, int NT, bool PD, bool STRIP = false>
__global__ void __launch_bounds__(NT, STRIP ? (NT == 128 ? 4 : 2) : (NT == 128 ? 6 : 3)) k_persist(Dev d, const int2 *__restrict__ tiles, int ntiles,
                                                                   int TR, int RS, int nintra, long long limit_ns) {
    extern __shared__ __align__(16) int smem[];
    __shared__ StepPlan sP;
    __shared__ int s_go, s_ok, s_app;
    Control *C = d.ctl;
    const int tid = threadIdx.x, G = gridDim.x, cta = blockIdx.x;
    const int nw = blockDim.x >> 5, warp = tid >> 5, lane = tid & 31;
    const int TC = (STRIP ? nw : nw / RS) * 32;
    const int items = STRIP ? nintra : ntiles + nintra;
    unsigned long long target = 0;
    bool ok = true;
    if (tid == 0) s_go = *(volatile int *)&C->done == 0;  // later steps learn of a stop at the barrier
    __syncthreads();
    for (int step = 1; s_go; ++step) {
        // ---- evaluation (every CTA)
        int best = kBestInit;
        unsigned bidx = 0xffffffffu;
        // intra-route items first: their dependent loads take longest
        for (int t = cta; t < items; t += G) {
            if (!STRIP && t >= nintra) {
                const int2 tl = tile_of(t - nintra, d.Wp, TR, TC);
                inter_tile<TW, OR, PD>(d, tl.x * TR, tl.y * TC, TR, RS, smem, best, bidx);
            } else if (TW) {
                __syncthreads();                       // smem of the previous item is free
                intra_route_table<PD>(d, t, smem, best, bidx);
            } else if (d.cvrp_by_route) {
                __syncthreads();
                intra_cvrp_route(d, t * nw + warp, lane, smem + warp * kCvrpRouteInts,
                                 smem + nw * kCvrpRouteInts + warp * 32, best, bidx);
            } else {
                intra_cvrp_position(d, t * nw + warp, lane, best, bidx);
            }
        }
        if (STRIP)
            strip_walk<TW, OR, PD>(d, TR, ntiles, (long long)cta * ntiles / G, (long long)(cta + 1) * ntiles / G,
                                   smem, best, bidx);
        const unsigned long long key = (bidx != 0xffffffffu) ? pack_key(best, bidx) : kNoKey;
        block_min_to(key, &C->best_key);
        // ---- the last CTA to finish decodes and publishes the plan, then
        // applies it itself; every other CTA waits for the publication (this
        // wait stands in for a barrier) and permutes distance columns
        if (tid == 0) {
            s_ok = 0;
            // release: this CTA's key is folded in; acquire: so are all the others'
            if (atom_add_acq_rel(&C->eval_done, 1) == G - 1) {
                C->eval_done = 0;
                decode_plan(d, nullptr, sP);
                C->plan = sP;
                C->plan_cta = cta;
                st_release(&C->plan_seq, step);        // publishes the plan
                s_ok = 1;
                s_app = cta;
            } else {
                s_ok = wait_seq(&C->plan_seq, step, limit_ns) ? 2 : 0;
                if (s_ok) s_app = *(volatile int *)&C->plan_cta;
            }
        }
        __syncthreads();
        if (!s_ok) { ok = false; break; }
        if (s_ok == 2) load_plan(C, &sP);
        __syncthreads();
        // ---- update
        int stop = 0;                                  // thread 0 of the applying CTA
        if (s_ok == 1) {
            stop = apply_plan_block<PD>(d, sP, smem, false, 0, 0);
            if (G == 1) {
                __syncthreads();
                band_plan_rows(d, sP, smem, 0, d.n + 1, 0, 1);
            }
        } else {
            band_plan_rows(d, sP, smem, 0, d.n + 1, cta < s_app ? cta : cta - 1, G - 1);
        }
        target += G;
        const int passed = grid_barrier(&C->bar_count, target, tid == 0 && stop != 0, limit_ns);
        if (!passed) { ok = false; break; }
        if (passed == 2) break;
    }
    if (!ok) {
        if (tid == 0) {
            set_status(C, TGA_ERR_TIMEOUT);
            __threadfence();                           // the status is visible before the stop flag
            C->done = 1;
        }
        return;
    }
    // the caller's solution is written back by the launch that follows
    // (k_sync_solution), which sees the final status of every CTA
}

namespace {

using PersistFn = void (*)(Dev, const int2 *, int, int, int, int, long long);

template <int NT, bool S>
PersistFn persist_fn_t(bool tw, bool orr, bool pd) {
    if (pd) return orr ? k_persist<true, true, NT, true, S> : k_persist<true, false, NT, true, S>;
    if (tw) return orr ? k_persist<true, true, NT, false, S> : k_persist<true, false, NT, false, S>;
    return orr ? k_persist<false, true, NT, false, S> : k_persist<false, false, NT, false, S>;
}

PersistFn persist_fn(bool tw, bool orr, int nt, bool pd, bool strip) {
    if (strip) return nt == 128 ? persist_fn_t<128, true>(tw, orr, pd) : persist_fn_t<256, true>(tw, orr, pd);
    return nt == 128 ? persist_fn_t<128, false>(tw, orr, pd) : persist_fn_t<256, false>(tw, orr, pd);
}

}  // namespace

int launch_persist(const Dev &d, const int2 *tiles, int ntiles, int rows, int warps, int rs, cudaStream_t s,
                   int *grid_out) {
    const bool strip = rs == 0;                           // strip-major walk of the ntiles tiles
    const int nt = warps * 32 * (strip ? 1 : rs);
    if (d.theta > 0) return TGA_ERR_STATE;                // edge-based extraction: per-step path only
    if (d.op_mask & kExtOps) return TGA_ERR_STATE;        // swaps of runs: per-step path only
    if (ntiles <= 0 || (nt != 128 && nt != 256)) return TGA_ERR_INVALID;   // apply needs >= 3 warps
    if (strip && !((rows == 16 || rows == 32) && (warps == 4 || warps == 8))) return TGA_ERR_INVALID;
    const int nw = nt / 32;
    const bool tw = d.has_tw != 0, orr = (d.op_mask & 48u) != 0, pd = d.has_pd != 0;
    const int nintra = tw ? d.m : d.cvrp_by_route ? (d.m + nw - 1) / nw : (d.Wp - 1 + nw - 1) / nw;
    size_t sm = strip ? strip_smem_bytes(rows, warps, pd) : inter_smem_bytes(rows, warps, pd);
    const size_t cvrp_intra = (size_t)nw * (kCvrpRouteInts + 32) * sizeof(int);
    if (!tw && d.cvrp_by_route && cvrp_intra > sm) sm = cvrp_intra;
    const size_t band = (size_t)band_smem_ints(d.Wp, nw) * sizeof(int);
    if (band > sm) sm = band;
    const size_t tab = (size_t)(pd ? kIntraTabSmemIntsPD : kIntraTabSmemInts) * sizeof(int);
    if (tw && tab > sm) sm = tab;
    if (sm > 200 * 1024) return TGA_ERR_RANGE;
    PersistFn fn = persist_fn(tw, orr, nt, pd, strip);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
        cudaGetLastError();
        return TGA_ERR_CUDA;
    }
    int dev = 0, nsm = 0, per = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return TGA_ERR_STATE;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, nt, sm) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return TGA_ERR_RANGE;
    }
    long long G = (long long)per * nsm;
    const long long items = (long long)ntiles + nintra;
    if (G > items) G = items;
    if (G < 1) G = 1;
    Dev dd = d;
    const int2 *tp = tiles;
    int nti = ntiles, tr = rows, rsv = rs, ni = nintra;
    long long limit = wait_limit(d.wait_ns, kWaitPersistNs);
    void *args[] = {&dd, &tp, &nti, &tr, &rsv, &ni, &limit};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void *)fn, dim3((unsigned)G), dim3((unsigned)nt), args,
                                                      sm, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TGA_ERR_CUDA;
    }
    if (grid_out) *grid_out = (int)G;
    return TGA_OK;
}

}  // namespace tga
