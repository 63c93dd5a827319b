// Batched descent: many independent instances in one persistent launch.
//
// Every job (context) is split, per local-search step, into chunks: one
// chunk per row tile of its inter-route pair triangle and one per group of
// eight routes for the intra-route moves.  Resident CTAs take chunks of any
// job from the job's counter, fold the chunk's candidates into the job's
// packed best key, and count the chunk as done; the CTA that completes a
// job's last chunk of a step applies that step's best move (the same device
// functions as the single-instance path) and then releases the job's next
// step.  Big jobs therefore spread over many SMs while small jobs finish in
// a few chunks, and no CTA ever waits for another: a CTA that finds no free
// chunk only polls again, under a time limit that reports TGA_ERR_TIMEOUT.
//
// Jobs are built inside the same launch (one CTA per job) before their
// chunks are released.  Compiled with L1 caching of global loads disabled,
// since a job's state is rewritten by whichever SM applied the last move.
#define TGA_LDG(p) (*(p))
#include "tga_device.cuh"
#undef TGA_FILE_ID
#define TGA_FILE_ID 5

namespace tga {

namespace {

// Build one job with the whole block (positions, validation, attributes of
// every route, the position-ordered distance copy), then arm its step limit.
__device__ void build_job(const Dev &d, long long max_steps) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    check_instance_tiles(d, 0, 1);
    __syncthreads();
    for (int x = tid; x <= d.n; x += nthr) d.seen[TGA_IX(x, d.n + 1)] = 0;
    __syncthreads();
    for (int r = tid; r < d.m; r += nthr) build_positions_route(d, r);
    __syncthreads();
    for (int x = tid + 1; x <= d.n; x += nthr) check_perm_one(d, x);
    __syncthreads();
    const int st = *(volatile int *)&d.ctl->status;
    if (st == 0)
        for (int r = warp; r < d.m; r += nw) rebuild_route<false>(d, r, lane);
    __syncthreads();
    finish_block(d);
    __syncthreads();
    pcol_init_range(d, tid, nthr);
    __syncthreads();
    if (tid == 0) {
        Control *C = d.ctl;
        C->step_limit = max_steps;
        if (C->status != 0) C->done = 1;
    }
    __syncthreads();
}

// Evaluation chunk c of a job.  c < ninter: row tiles chunk_t0[c] ..
// chunk_t0[c+1]-1 of its pair triangle; a job with a single such chunk also
// evaluates all its intra-route moves there (a small job's whole step in one
// chunk).  Larger jobs get separate intra chunks: 8 routes (VRPTW) or 8 moved
// positions (CVRP) each, so long routes spread over many SMs.
template <bool TW>
__device__ void run_chunk(const BatchJob &J, int c, int *smem, int &best, unsigned &bidx) {
    const Dev &d = J.d;
    const bool OR = (d.op_mask & 48u) != 0;
    const int TC = blockDim.x, TR = J.tr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int r_lo = 0, r_hi = 0, p_lo = 0, p_hi = 0;
    if (c < J.ninter) {
        const int t0 = J.chunk_t0[c], t1 = J.chunk_t0[c + 1];
        for (int I = t0; I < t1; ++I) {
            const long long j0 = ((long long)I * TR + 1) / TC;     // first J with (J+1)*TC-1 > I*TR
            for (int Jc = (int)j0; Jc < J.nct; ++Jc) {
                if (OR) inter_tile<TW, true>(d, I * TR, Jc * TC, TR, 1, smem, best, bidx);
                else inter_tile<TW, false>(d, I * TR, Jc * TC, TR, 1, smem, best, bidx);
            }
        }
        if (J.ninter > 1) return;
        r_hi = d.m;
        p_hi = d.Wp - 1;
    } else {
        const int g = c - J.ninter;
        r_lo = g * nw; r_hi = min(r_lo + nw, d.m);
        p_lo = g * nw; p_hi = min(p_lo + nw, d.Wp - 1);
    }
    __syncthreads();
    if (!TW) {
        for (int p = p_lo + warp; p < p_hi; p += nw) intra_cvrp_position(d, p, lane, best, bidx);
    } else {
        for (int r = r_lo + warp; r < r_hi; r += nw)
            intra_route<TW>(d, r, lane, smem + warp * kIntraSmemPerWarp, best, bidx);
    }
}

// A job is finished: write its solution back (when moves may have been
// applied) and count it (whole block).
__device__ void finish_job(const Dev &d, BatchState *B, bool write_solution) {
    if (write_solution) sync_solution_range(d, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        d.ctl->finished = 1;
        __threadfence();
        atomicAdd(&B->jobs_done, 1);
    }
}

// Open the job's next evaluation (one thread).
__device__ void release_eval(Control *C) {
    C->done_chunks = 0;
    __threadfence();
    atomicExch(&C->next_chunk, 0);
}

}  // namespace

__global__ void k_batch_init(const BatchJob *jobs, int njobs, BatchState *B) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) { B->build_next = 0; B->jobs_done = 0; B->status = 0; B->pad = 0; }
    if (j >= njobs) return;
    Control *C = jobs[j].d.ctl;
    C->next_chunk = 0x3fffffff;                 // no chunk before the job is built
    C->done_chunks = 0;
    C->band_next = 0x3fffffff;
    C->band_done = 0;
    C->finished = 0;
}

// Copy job j's descriptor into shared memory (the device functions read its
// fields constantly; immutable for the whole launch).
__device__ __forceinline__ void load_job(const BatchJob *jobs, int j, BatchJob *sJ) {
    const int words = (int)(sizeof(BatchJob) / sizeof(int));
    const int *src = reinterpret_cast<const int *>(jobs + j);
    int *dst = reinterpret_cast<int *>(sJ);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

__global__ void __launch_bounds__(kBatchThreads) k_batch(const BatchJob *__restrict__ jobs, int njobs,
                                                         BatchState *B, long long max_steps, int mode,
                                                         long long idle_limit_ns) {
    extern __shared__ __align__(16) int smem[];
    __shared__ __align__(16) BatchJob sJ;
    __shared__ int s_j, s_c, s_ph, s_last, s_stop;
    __shared__ StepPlan sPlan;
    const int tid = threadIdx.x;
    const bool eval_only = mode != 0;

    // ---- build: one job per CTA at a time
    for (;;) {
        if (tid == 0) s_j = atomicAdd(&B->build_next, 1);
        __syncthreads();
        const int j = s_j;
        __syncthreads();
        if (j >= njobs) break;
        load_job(jobs, j, &sJ);
        if (mode != 2) {
            build_job(sJ.d, max_steps);
        } else if (tid == 0) {
            sJ.d.ctl->best_key = kNoKey;
        }
        if (tid == 0) {
            Control *C = sJ.d.ctl;
            __threadfence();
            if (C->status != 0 || max_steps <= 0) {
                C->finished = 1;
                atomicAdd(&B->jobs_done, 1);
            } else {
                atomicExch(&C->next_chunk, 0);
            }
        }
        __syncthreads();
    }

    // ---- descend: take chunks of any job until every job is finished
    int start = blockIdx.x % njobs;
    long long idle_since = -1;
    int cached = -1;                                  // job whose descriptor sJ holds
    for (;;) {
        if (tid == 0) {
            s_j = -1;
            s_stop = (*(volatile int *)&B->jobs_done >= njobs) || (*(volatile int *)&B->status != 0);
            if (!s_stop) {
                for (int k = 0; k < njobs; ++k) {
                    const int jj = (start + k) % njobs;
                    Control *C = jobs[jj].d.ctl;
                    const int nch = jobs[jj].nchunks, nb = jobs[jj].nband;
                    if (*(volatile int *)&C->next_chunk < nch) {
                        const int c = atomicAdd(&C->next_chunk, 1);
                        if (c < nch) { s_j = jj; s_c = c; s_ph = 0; break; }
                    } else if (*(volatile int *)&C->band_next < nb) {
                        const int c = atomicAdd(&C->band_next, 1);
                        if (c < nb) { s_j = jj; s_c = c; s_ph = 1; break; }
                    }
                }
                if (s_j < 0) {
                    const long long t = now_ns();
                    if (idle_since < 0) idle_since = t;
                    else if (t - idle_since > idle_limit_ns) {
                        atomicCAS(&B->status, 0, TGA_ERR_TIMEOUT);
                        s_stop = 1;
                    }
                } else {
                    idle_since = -1;
                }
            }
        }
        __syncthreads();
        if (s_stop) break;
        const int jj = s_j, c = s_c, ph = s_ph;
        if (jj < 0) {
            __nanosleep(256);
            __syncthreads();
            continue;
        }
        start = jj;
        __threadfence();   // acquire the job state released with the chunk counter
        if (jj != cached) {
            load_job(jobs, jj, &sJ);
            cached = jj;
        }
        const BatchJob &J = sJ;
        Control *C = J.d.ctl;
        if (ph == 1) {
            // column-permutation chunk of the move just applied
            load_plan(C, &sPlan);
            __syncthreads();
            band_plan_rows(J.d, sPlan, smem, c * kBandRowsPerChunk, (c + 1) * kBandRowsPerChunk, 0, 1);
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                s_last = atomicAdd(&C->band_done, 1) == J.nband - 1;
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                if (*(volatile int *)&C->done || C->steps >= C->step_limit) finish_job(J.d, B, true);
                else if (tid == 0) release_eval(C);
            }
            __syncthreads();
            continue;
        }
        int best = kBestInit;
        unsigned bidx = 0xffffffffu;
        if (J.d.has_tw) run_chunk<true>(J, c, smem, best, bidx);
        else run_chunk<false>(J, c, smem, best, bidx);
        const unsigned long long key = (bidx != 0xffffffffu) ? pack_key(best, bidx) : kNoKey;
        block_min_to(key, &C->best_key);
        if (tid == 0) {
            __threadfence();
            s_last = atomicAdd(&C->done_chunks, 1) == J.nchunks - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            const Dev &d = J.d;
            if (!eval_only) {
                if (tid == 0) {
                    decode_plan(d, nullptr, sPlan);
                    C->plan = sPlan;
                }
                __syncthreads();
                apply_plan_block<false>(d, sPlan, smem, false, 0, 0);
            } else if (tid == 0) {
                if (d.log && C->evals < d.log_cap) d.log[C->evals] = C->best_key;
                count_evaluation(d, C);
                sPlan.act = 0;
            }
            __syncthreads();
            if (sPlan.act) {
                if (tid == 0) {                        // release the permutation chunks
                    C->band_done = 0;
                    __threadfence();
                    atomicExch(&C->band_next, 0);
                }
            } else {
                finish_job(d, B, !eval_only);
            }
            __syncthreads();
        }
    }
}

size_t batch_smem_bytes(int max_tr, int max_wp) {
    size_t a = inter_smem_bytes(max_tr, kBatchThreads / 32);
    const size_t b = (size_t)(kBatchThreads / 32) * kIntraSmemPerWarp * sizeof(int);
    const size_t c = (size_t)band_smem_ints(max_wp, kBatchThreads / 32) * sizeof(int);
    if (b > a) a = b;
    if (c > a) a = c;
    return a;
}

int launch_batch(const BatchJob *jobs_dev, int njobs, BatchState *state_dev, long long max_steps, int mode,
                 int max_tr, int max_wp, long long idle_limit_ns, cudaStream_t s) {
    const size_t sm = batch_smem_bytes(max_tr, max_wp);
    if (sm > 200 * 1024) return TGA_ERR_RANGE;
    if (cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return TGA_ERR_CUDA;
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, kBatchThreads, sm);
    if (per < 1) return TGA_ERR_RANGE;
    const int grid = nsm * per;
    k_batch_init<<<(njobs + 127) / 128, 128, 0, s>>>(jobs_dev, njobs, state_dev);
    k_batch<<<grid, kBatchThreads, sm, s>>>(jobs_dev, njobs, state_dev, max_steps, mode, idle_limit_ns);
    return cudaGetLastError() == cudaSuccess ? TGA_OK : TGA_ERR_CUDA;
}

}  // namespace tga
