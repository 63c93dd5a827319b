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
// count reaches k * G.  One thread per CTA waits, at most limit_ns.
__device__ bool grid_barrier(unsigned long long *count, unsigned long long target, long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        red_add_release(count, 1ull);                  // publishes the block's writes
        int ok = 1;
        if (ld_acquire(count) < target) {
            const long long t0 = now_ns();
            while (ld_acquire(count) < target) {
                if (now_ns() - t0 > limit_ns) { ok = 0; break; }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
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
// blockDim/32 moved positions per item (one warp each).
// PD: pickups (with time windows).
template <bool TW, bool OR, int NT, bool PD>
__global__ void __launch_bounds__(NT, NT == 128 ? 6 : 3) k_persist(Dev d, const int2 *__restrict__ tiles, int ntiles,
                                                                   int TR, int RS, int nintra, long long limit_ns) {
    extern __shared__ __align__(16) int smem[];
    __shared__ StepPlan sP;
    __shared__ int s_go, s_ok, s_app;
    Control *C = d.ctl;
    const int tid = threadIdx.x, G = gridDim.x, cta = blockIdx.x;
    const int nw = blockDim.x >> 5, warp = tid >> 5, lane = tid & 31;
    const int TC = (nw / RS) * 32;
    const int items = ntiles + nintra;
    unsigned long long target = 0;
    bool ok = true;
    for (int step = 1;; ++step) {
        if (tid == 0) s_go = *(volatile int *)&C->done == 0;
        __syncthreads();
        if (!s_go) break;
        // ---- evaluation (every CTA)
        int best = kBestInit;
        unsigned bidx = 0xffffffffu;
        // intra-route items first: their dependent loads take longest
        for (int t = cta; t < items; t += G) {
            if (t >= nintra) {
                const int2 tl = tile_of(t - nintra, d.Wp, TR, TC);
                inter_tile<TW, OR, PD>(d, tl.x * TR, tl.y * TC, TR, RS, smem, best, bidx);
            } else if (TW) {
                __syncthreads();                       // smem of the previous item is free
                intra_route_table<PD>(d, t, smem, best, bidx);
            } else {
                intra_cvrp_position(d, t * nw + warp, lane, best, bidx);
            }
        }
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
        if (s_ok == 1) {
            apply_plan_block<PD>(d, sP, smem, false, 0, 0);
            if (G == 1) {
                __syncthreads();
                band_plan_rows(d, sP, smem, 0, d.n + 1, 0, 1);
            }
        } else {
            band_plan_rows(d, sP, smem, 0, d.n + 1, cta < s_app ? cta : cta - 1, G - 1);
        }
        target += G;
        if (!grid_barrier(&C->bar_count, target, limit_ns)) { ok = false; break; }
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

PersistFn persist_fn(bool tw, bool orr, int nt, bool pd) {
    if (nt == 128) {
        if (pd) return orr ? k_persist<true, true, 128, true> : k_persist<true, false, 128, true>;
        if (tw) return orr ? k_persist<true, true, 128, false> : k_persist<true, false, 128, false>;
        return orr ? k_persist<false, true, 128, false> : k_persist<false, false, 128, false>;
    }
    if (pd) return orr ? k_persist<true, true, 256, true> : k_persist<true, false, 256, true>;
    if (tw) return orr ? k_persist<true, true, 256, false> : k_persist<true, false, 256, false>;
    return orr ? k_persist<false, true, 256, false> : k_persist<false, false, 256, false>;
}

}  // namespace

int launch_persist(const Dev &d, const int2 *tiles, int ntiles, int rows, int warps, int rs, cudaStream_t s,
                   int *grid_out) {
    const int nt = warps * 32 * rs;
    if (d.theta > 0) return TGA_ERR_STATE;                // edge-based extraction: per-step path only
    if (d.op_mask & kExtOps) return TGA_ERR_STATE;        // swaps of runs: per-step path only
    if (ntiles <= 0 || (nt != 128 && nt != 256)) return TGA_ERR_INVALID;   // apply needs >= 3 warps
    const int nw = nt / 32;
    const bool tw = d.has_tw != 0, orr = (d.op_mask & 48u) != 0, pd = d.has_pd != 0;
    const int nintra = tw ? d.m : (d.Wp - 1 + nw - 1) / nw;
    size_t sm = inter_smem_bytes(rows, warps, pd);
    const size_t band = (size_t)band_smem_ints(d.Wp, nw) * sizeof(int);
    if (band > sm) sm = band;
    const size_t tab = (size_t)(pd ? kIntraTabSmemIntsPD : kIntraTabSmemInts) * sizeof(int);
    if (tw && tab > sm) sm = tab;
    if (sm > 200 * 1024) return TGA_ERR_RANGE;
    PersistFn fn = persist_fn(tw, orr, nt, pd);
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
