// libtga C-ABI: context lifetime, the descent loop as a CUDA graph with a
// device-driven conditional while node, and the tile-shape autotuner.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "tga_internal.cuh"

using namespace tga;

namespace {
// NVTX range around one entry point (host time: the enqueue for the
// asynchronous calls, the whole call for the synchronising ones).  The NVTX
// header is self-contained: without a profiler attached each range costs a
// function-pointer test.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
}  // namespace

struct tga_ctx {
    Dev d{};
    cudaStream_t stream = nullptr;     // caller's stream
    cudaStream_t cap = nullptr;        // private stream used only for graph capture
    cudaStream_t cap2 = nullptr;       // second capture stream: the intra-route branch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int device = 0;
    bool built = false;
    // inter-route tiles
    int tile_rows = 0, tile_warps = 0, tile_rs = 1, ntiles = 0;
    int strip = 0;                     // strip-major inter kernel: its grid (0: one CTA per tile)
    int2 *tiles = nullptr;
    std::vector<int2> tiles_host;      // kept alive for the asynchronous upload
    // descent graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ready = false;
    bool graph_failed = false;
    int batch_tr = 0;                  // tile rows in batched descents (0: by size)
    // descent path: requested mode and the one the last descent took
    int mode = TGA_DESCENT_AUTO;
    int last_mode = TGA_DESCENT_AUTO;
    int persist_grid = 0;
    // measured choice for the automatic mode (0: not measured, size rule)
    // and the persistent path's tile shape (0: derived from the inter tile)
    int auto_choice = 0;
    int ptile_rows = 0, ptile_warps = 0, ptile_rs = 0;
    int *saved = nullptr;              // workspace copy of the caller's solution (tuning)
    void *granular = nullptr;          // reverse-entry flags of the mask rows + a check word
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? TGA_OK : TGA_ERR_CUDA; }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int check_launch() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "libtga: CUDA error: %s\n", cudaGetErrorString(e));
        return TGA_ERR_CUDA;
    }
    return TGA_OK;
}

void drop_graph(tga_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->graph_ready = false;
}

// strip: run the tiles with the strip-major kernel (rows 16 or 32, 4 or 8
// warps, no row split).
int set_tiles(tga_ctx *c, int rows, int warps, int rs = 1, bool strip = false) {
    if (!(rows == 8 || rows == 16 || rows == 32 || rows == 64) || !(warps == 2 || warps == 4 || warps == 8) ||
        !(rs == 1 || rs == 2 || rs == 4) || warps * rs > 8 || rows % rs != 0)
        return TGA_ERR_INVALID;
    if (strip && (rs != 1 || !(rows == 16 || rows == 32) || !(warps == 4 || warps == 8))) return TGA_ERR_INVALID;
    const int Wa = c->d.Wp - 1;   // anchor positions
    const int TC = warps * 32;
    const int nrt = (Wa + rows - 1) / rows, nct = (Wa + TC - 1) / TC;
    std::vector<int2> &t = c->tiles_host;
    t.clear();
    t.reserve((size_t)nrt * nct / 2 + nrt + 8);
    for (int I = 0; I < nrt; ++I)
        for (int J = 0; J < nct; ++J)
            if ((long long)(J + 1) * TC - 1 > (long long)I * rows) t.push_back(make_int2(I, J));
    // stream-ordered allocation: no device-wide synchronisation, so other
    // contexts' work keeps running while this one is set up or torn down
    if (c->tiles) cudaFreeAsync(c->tiles, c->stream);
    c->tiles = nullptr;
    c->ntiles = (int)t.size();
    if (!t.empty()) {
        if (cudaMallocAsync((void **)&c->tiles, t.size() * sizeof(int2), c->stream) != cudaSuccess) {
            cudaGetLastError();
            return TGA_ERR_NOMEM;
        }
        if (cudaMemcpyAsync(c->tiles, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
            return TGA_ERR_CUDA;
    }
    c->tile_rows = rows;
    c->tile_warps = warps;
    c->tile_rs = rs;
    c->strip = strip ? strip_grid(c->d, rows, warps, c->ntiles) : 0;
    drop_graph(c);
    if (strip && c->ntiles > 0 && c->strip == 0) return TGA_ERR_CUDA;
    return TGA_OK;
}

// Shapes measured fastest on a GB300 before any autotuning: one CTA per
// 16 x 64 tile for small instances (a single wave), the strip-major kernel
// with 16-row tiles otherwise (column strips of 128 or 256 positions).
void default_tiles(tga_ctx *c) {
    const long long pairs = (long long)c->d.Wp * c->d.Wp / 2;
    if (pairs < 2000000) set_tiles(c, 16, 2);
    else if (pairs < 20000000) set_tiles(c, 16, 4, 1, true);
    else set_tiles(c, 16, 8, 1, true);
}

int step_once(tga_ctx *c, unsigned long long cond, int use_cond, cudaStream_t s) {
    launch_eval(c->d, c->tiles, c->ntiles, c->tile_rows, c->tile_warps, s, c->tile_rs,
                eval_blocks(c->d, c->ntiles, c->strip), c->strip);
    launch_apply(c->d, nullptr, cond, use_cond, s, 1);
    return check_launch();
}

int build_graph(tga_ctx *c) {
    if (c->graph_ready) return TGA_OK;
    if (c->graph_failed) return TGA_ERR_CUDA;
    cudaError_t e = cudaGraphCreate(&c->graph, 0);
    cudaGraphConditionalHandle h = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, c->graph, nullptr, nullptr, 0, &cp);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            // inter-route tiles and intra-route routes run as parallel
            // branches; both fold into the same packed best key
            cudaEventRecord(c->ev_fork, c->cap);
            cudaStreamWaitEvent(c->cap2, c->ev_fork, 0);
            const int tail = eval_blocks(c->d, c->ntiles, c->strip);
            launch_inter(c->d, c->tiles, c->ntiles, c->tile_rows, c->tile_warps, c->cap, c->tile_rs, tail, c->strip);
            launch_intra(c->d, c->cap2, tail);
            launch_xswap(c->d, c->cap2, tail);
            cudaEventRecord(c->ev_join, c->cap2);
            cudaStreamWaitEvent(c->cap, c->ev_join, 0);
            launch_apply(c->d, nullptr, h, 1, c->cap, 1);
            cudaGraph_t outg = body;
            e = cudaStreamEndCapture(c->cap, &outg);
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, c->graph, 0);
    if (e != cudaSuccess) {
        fprintf(stderr, "libtga: graph build failed (%s); using host-driven steps\n", cudaGetErrorString(e));
        cudaGetLastError();
        drop_graph(c);
        c->graph_failed = true;
        return TGA_ERR_CUDA;
    }
    c->graph_ready = true;
    return TGA_OK;
}

int read_control(tga_ctx *c, Control *out) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return TGA_ERR_CUDA;
    e = cudaMemcpyAsync(out, c->d.ctl, sizeof(Control), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_err(e);
}

void fill_stats(const Control &C, tga_stats *s) {
    s->steps = C.steps;
    s->candidates = C.cand_total;
    s->initial_cost = C.initial_cost;
    s->final_cost = C.cost;
    s->status = C.status;
    s->local_optimum = C.local_opt;
    s->evaluations = C.evals;
}

// Instances below this many positions descend in one persistent launch when
// the mode is automatic; larger ones run the per-step graph.
constexpr int kPersistAutoMaxWp = 4096;

// Persistent descent with the context's tile shape; the row split is raised
// until a block has at least 4 warps (the tile list does not depend on it).
long long count_tiles(int Wp, int rows, int TC) {
    const long long Wa = Wp - 1, nrt = (Wa + rows - 1) / rows, nct = (Wa + TC - 1) / TC;
    long long t = 0;
    for (long long I = 0; I < nrt; ++I) {
        const long long j0 = (I * rows + 1) / TC;            // first J with (J+1)*TC-1 > I*rows
        t += nct > j0 ? nct - j0 : 0;
    }
    return t;
}

int persist_shape(int rows, int warps, int rs, const Dev &d, cudaStream_t s, int *grid) {
    return launch_persist(d, nullptr, (int)count_tiles(d.Wp, rows, warps * 32), rows, warps, rs, s, grid);
}

int try_persist(tga_ctx *c) {
    if (c->ptile_rows)
        return persist_shape(c->ptile_rows, c->ptile_warps, c->ptile_rs, c->d, c->stream, &c->persist_grid);
    int rs = c->tile_rs;
    while (c->tile_warps * 32 * rs < 128 && rs < 4 && c->tile_warps * rs * 2 <= 8 && c->tile_rows % (rs * 2) == 0)
        rs *= 2;
    return launch_persist(c->d, c->tiles, c->ntiles, c->tile_rows, c->tile_warps, rs, c->stream, &c->persist_grid);
}

int descend_launch(tga_ctx *c, int64_t max_steps) {
    if (!c->built) {
        int rc = tga_build_attrs(c);
        if (rc) return rc;
    }
    if (!c->tiles && c->d.Wp > 2) default_tiles(c);
    launch_begin(c->d, max_steps, c->stream);
    if (max_steps == 0) return check_launch();       // the graph body runs at least once
    int mode = c->mode;
    // TGA_GRAPH=0 launches the per-step kernels from the host (for profilers
    // that do not trace kernels inside conditional graph bodies)
    const char *env = getenv("TGA_GRAPH");
    if (env && env[0] == '0') mode = TGA_DESCENT_HOST;
    const bool automatic = mode == TGA_DESCENT_AUTO;
    if (automatic)
        mode = c->auto_choice ? c->auto_choice
                              : (c->d.Wp < kPersistAutoMaxWp ? TGA_DESCENT_PERSISTENT : TGA_DESCENT_GRAPH);
    if (mode == TGA_DESCENT_PERSISTENT) {
        const int rc = try_persist(c);
        if (rc == TGA_OK) {
            launch_sync_solution(c->d, c->stream);
            c->last_mode = TGA_DESCENT_PERSISTENT;
            return check_launch();
        }
        if (!automatic) return rc;
        mode = TGA_DESCENT_GRAPH;
    }
    if (mode == TGA_DESCENT_GRAPH && build_graph(c) == TGA_OK) {
        if (cudaGraphLaunch(c->gexec, c->stream) != cudaSuccess) return TGA_ERR_CUDA;
        launch_sync_solution(c->d, c->stream);
        c->last_mode = TGA_DESCENT_GRAPH;
        return check_launch();
    }
    c->last_mode = TGA_DESCENT_HOST;
    // host-driven fallback: chunks of steps, stop when the device says done
    Control C;
    int64_t done_steps = 0;
    while (done_steps < max_steps) {
        const int chunk = 64;
        for (int k = 0; k < chunk; ++k) {
            int rc = step_once(c, 0, 0, c->stream);
            if (rc) return rc;
        }
        done_steps += chunk;
        int rc = read_control(c, &C);
        if (rc) return rc;
        if (C.done) break;
    }
    launch_sync_solution(c->d, c->stream);
    return check_launch();
}

int default_batch_tr(int Wp) { return Wp < 600 ? 16 : (Wp < 2000 ? 32 : 64); }

// One persistent launch over all contexts (see tga_batch.cu).
int run_batch(tga_ctx **ctxs, int n, long long max_steps, int mode, const int *tr_override) {
    for (int i = 0; i < n; ++i)                  // no edge-based or pickup path in the batched kernel
        if (ctxs[i]->d.theta > 0 || ctxs[i]->d.has_pd || (ctxs[i]->d.op_mask & kExtOps)) return TGA_ERR_STATE;
    cudaStream_t s = ctxs[0]->stream;
    for (int i = 0; i < n; ++i)
        if (ctxs[i]->stream != s && cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) return TGA_ERR_CUDA;
    std::vector<BatchJob> jobs((size_t)n);
    std::vector<std::vector<int>> bounds((size_t)n);
    int max_tr = 16, max_wp = 1;
    size_t nbounds = 0;
    long long idle_ns = kWaitBatchNs;
    for (int i = 0; i < n; ++i) {
        tga_ctx *c = ctxs[i];
        const int tr = tr_override ? tr_override[i] : (c->batch_tr ? c->batch_tr : default_batch_tr(c->d.Wp));
        BatchJob &J = jobs[(size_t)i];
        J.d = c->d;
        J.tr = tr;
        const int Wa = c->d.Wp - 1;
        J.nrt = (Wa + tr - 1) / tr;
        J.nct = (Wa + kBatchThreads - 1) / kBatchThreads;
        // group consecutive row tiles into chunks of about kChunkPairs pairs
        std::vector<int> &b = bounds[(size_t)i];
        b.push_back(0);
        long long acc = 0;
        for (int I = 0; I < J.nrt; ++I) {
            const long long j0 = ((long long)I * tr + 1) / kBatchThreads;   // first J with (J+1)*TC-1 > I*tr
            acc += (long long)(J.nct - j0) * tr * kBatchThreads;
            if (acc >= kChunkPairs && I + 1 < J.nrt) { b.push_back(I + 1); acc = 0; }
        }
        b.push_back(J.nrt);
        J.ninter = (int)b.size() - 1;
        const int nw = kBatchThreads / 32;
        const int nintra = J.ninter == 1 ? 0 : ((c->d.has_tw ? c->d.m : Wa) + nw - 1) / nw;
        J.nchunks = J.ninter + nintra;
        J.nband = (c->d.n + 1 + kBandRowsPerChunk - 1) / kBandRowsPerChunk;
        J.chunk_t0 = nullptr;
        nbounds += b.size();
        if (tr > max_tr) max_tr = tr;
        idle_ns = std::min(idle_ns, wait_limit(c->d.wait_ns, kWaitBatchNs));
        if (c->d.Wp > max_wp) max_wp = c->d.Wp;
        if (mode != 2 && cudaMemsetAsync(c->d.ctl, 0, sizeof(Control), s) != cudaSuccess) return TGA_ERR_CUDA;
    }
    // largest jobs first: their chunks are taken before the small jobs'
    std::vector<BatchJob> ordered(jobs);
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return jobs[(size_t)a].d.Wp > jobs[(size_t)b].d.Wp; });
    for (int i = 0; i < n; ++i) ordered[(size_t)i] = jobs[(size_t)order[(size_t)i]];
    char *buf = nullptr;
    const size_t jb = align_up(sizeof(BatchJob) * (size_t)n, 256);
    const size_t sb = align_up(sizeof(BatchState), 256);
    if (cudaMalloc(&buf, jb + sb + sizeof(int) * nbounds) != cudaSuccess) { cudaGetLastError(); return TGA_ERR_NOMEM; }
    BatchJob *jdev = (BatchJob *)buf;
    BatchState *sdev = (BatchState *)(buf + jb);
    int *bdev = (int *)(buf + jb + sb);
    std::vector<int> flat;
    flat.reserve(nbounds);
    for (int i = 0; i < n; ++i) {
        BatchJob &J = ordered[(size_t)i];
        const std::vector<int> &b = bounds[(size_t)order[(size_t)i]];
        J.chunk_t0 = bdev + flat.size();
        flat.insert(flat.end(), b.begin(), b.end());
    }
    int rc = TGA_OK;
    if (cudaMemcpyAsync(jdev, ordered.data(), sizeof(BatchJob) * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(bdev, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = TGA_ERR_CUDA;
    if (!rc) rc = launch_batch(jdev, n, sdev, max_steps, mode, max_tr, max_wp, idle_ns, s);
    BatchState st{};
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = rc ? rc : TGA_ERR_CUDA;
    if (cudaMemcpy(&st, sdev, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) rc = rc ? rc : TGA_ERR_CUDA;
    cudaFree(buf);
    if (!rc && st.status) rc = st.status;
    // a failed launch may stop jobs mid-step: rebuild them on their next use
    if (mode != 2)
        for (int i = 0; i < n; ++i) ctxs[i]->built = rc == TGA_OK;
    return rc;
}

}  // namespace

// Mean milliseconds per launch of one evaluation kernel on the current state
// (`launch` issues it on the context's stream); leaves no pending key and the
// context's done flag as it was.
template <class F>
static int profile_launches(tga_ctx *c, int32_t reps, float *ms_per_launch, F launch) {
    Control C;
    int rc = read_control(c, &C);
    if (rc) return rc;
    const int was_done = C.done;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TGA_ERR_CUDA;
    // the kernels return immediately on a finished context: clear the flag
    cudaMemsetAsync(&c->d.ctl->done, 0, sizeof(int), c->stream);
    launch();                                                    // warm-up
    cudaEventRecord(e0, c->stream);
    for (int k = 0; k < reps; ++k) launch();
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_launch = ms / reps;
    cudaMemsetAsync(&c->d.ctl->best_key, 0xff, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(&c->d.ctl->done, 0, sizeof(int), c->stream);
    if (was_done) {
        int one = 1;
        cudaMemcpyAsync(&c->d.ctl->done, &one, sizeof(int), cudaMemcpyHostToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
    }
    return check_launch();
}

extern "C" {

const char *tga_strerror(int code) {
    switch (code) {
        case TGA_OK: return "ok";
        case TGA_ERR_INVALID: return "invalid argument, instance, solution or move";
        case TGA_ERR_RANGE: return "integer range or move-index bound exceeded";
        case TGA_ERR_NOMEM: return "device allocation failed";
        case TGA_ERR_CUDA: return "CUDA runtime error";
        case TGA_ERR_TIMEOUT: return "bounded device wait expired";
        case TGA_ERR_STATE: return "call not allowed in the current state";
        case TGA_ERR_CHECK: return "internal consistency check failed (applied delta differs from evaluated delta)";
        case TGA_ERR_BOUNDS: return "device index check failed (index-checked build)";
        default: return "unknown error";
    }
}

int tga_create(const tga_instance *inst, const tga_solution *sol, uint32_t op_mask, tga_stream_t stream,
               tga_ctx **out) {
    if (!inst || !sol || !out) return TGA_ERR_INVALID;
    *out = nullptr;
    const long long n = inst->n_customers, m = inst->n_routes;
    if (n < 1 || m < 1 || inst->capacity < 0 || inst->w_load < 0 || inst->w_tw < 0) return TGA_ERR_INVALID;
    if (op_mask == 0 || op_mask >= 256u) return TGA_ERR_INVALID;
    if (!inst->dist || !inst->demand || !sol->tour || !sol->route_start) return TGA_ERR_INVALID;
    if (inst->has_tw && (!inst->service || !inst->tw_early || !inst->tw_late)) return TGA_ERR_INVALID;
    if (inst->pickup && !inst->has_tw) return TGA_ERR_INVALID;       // pickups come with time windows
    if (inst->pickup && (op_mask & kExtOps)) return TGA_ERR_INVALID;  // no pickup variant of the run swaps
    const long long W = n + 1 + m;
    if (W > ((op_mask & kExtOps) ? kMaxWExt : kMaxW)) return TGA_ERR_RANGE;

    tga_ctx *c = new (std::nothrow) tga_ctx();
    if (!c) return TGA_ERR_NOMEM;
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        if (c->cap) cudaStreamDestroy(c->cap);
        if (c->cap2) cudaStreamDestroy(c->cap2);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        delete c;
        return TGA_ERR_CUDA;
    }
    Dev &d = c->d;
    d.n = (int)n; d.m = (int)m; d.W = (int)W; d.Wp = (int)(n + m + 1);
    d.Q = inst->capacity; d.wL = inst->w_load; d.wT = inst->w_tw; d.has_tw = inst->has_tw ? 1 : 0;
    d.has_pd = inst->pickup ? 1 : 0;
    d.op_mask = op_mask;
    d.dist = inst->dist; d.demand = inst->demand;
    d.service = inst->service; d.early = inst->tw_early; d.late = inst->tw_late;
    d.pickup = inst->pickup;
    d.tour = sol->tour; d.route_start = sol->route_start;
    d.cvrp_by_route = cvrp_intra_by_route(d.n, d.m, d.has_tw, d.op_mask);
    d.ldp = (int)pcol_pitch((size_t)d.Wp);
    d.log = nullptr; d.log_cap = 0;
    d.wait_ns = -1;
    if (cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || d.nsm < 1) {
        cudaGetLastError();
        tga_destroy(c);
        return TGA_ERR_CUDA;
    }

    const WsLayout L = workspace_layout((size_t)n, (size_t)m, d.has_pd != 0, (op_mask & kExtOps) != 0);
    c->ws_bytes = L.bytes;
    if (cudaMallocAsync(&c->ws, c->ws_bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        tga_destroy(c);
        return TGA_ERR_NOMEM;
    }
    char *base = (char *)c->ws;
    d.ctl = (Control *)(base + L.ctl);
    d.seq = (int *)(base + L.seq);
    d.pos_of = (int *)(base + L.pos);
    d.brec = (BRec *)(base + L.brec);
    d.erec = (ERec *)(base + L.erec);
    d.prec = d.has_pd ? (PRec *)(base + L.prec) : nullptr;
    d.xrec = (op_mask & kExtOps) ? (XRec *)(base + L.xrec) : nullptr;
    d.rrec = (RouteRec *)(base + L.rrec);
    d.seen = (int *)(base + L.seen);
    d.scr_intra = (int *)(base + L.intra);
    d.pcol = (int *)(base + L.pcol);
    c->saved = (int *)(base + L.saved);
    if (cudaMemsetAsync(d.ctl, 0, sizeof(Control), c->stream) != cudaSuccess ||
        setup_kernel_attrs(d.Wp) != 0) {
        tga_destroy(c);
        return TGA_ERR_CUDA;
    }
    *out = c;
    return TGA_OK;
}

int tga_build_attrs(tga_ctx *c) {
    const Range range("tga_build_attrs");
    if (!c) return TGA_ERR_INVALID;
    if (cudaMemsetAsync(c->d.ctl, 0, sizeof(Control), c->stream) != cudaSuccess) return TGA_ERR_CUDA;
    launch_check_instance(c->d, c->stream);
    launch_build(c->d, c->stream);
    c->built = true;
    return check_launch();
}

int tga_eval_best_move(tga_ctx *c, tga_move *out_dev) {
    const Range range("tga_eval_best_move");
    if (!c || !out_dev) return TGA_ERR_INVALID;
    if (!c->built) return TGA_ERR_STATE;
    if (!c->tiles && c->d.Wp > 2) default_tiles(c);
    launch_begin(c->d, 1, c->stream);
    launch_eval(c->d, c->tiles, c->ntiles, c->tile_rows, c->tile_warps, c->stream, c->tile_rs, 0, c->strip);
    launch_finalize(c->d, out_dev, c->stream);
    return check_launch();
}

int tga_apply_move(tga_ctx *c, const tga_move *move_dev) {
    const Range range("tga_apply_move");
    if (!c || !move_dev) return TGA_ERR_INVALID;
    if (!c->built) return TGA_ERR_STATE;
    launch_apply(c->d, move_dev, 0, 0, c->stream);
    launch_sync_solution(c->d, c->stream);
    return check_launch();
}

int tga_descend(tga_ctx *c, int64_t max_steps, tga_stats *out_host) {
    const Range range("tga_descend");
    if (!c || max_steps < 0) return TGA_ERR_INVALID;
    int rc = descend_launch(c, max_steps);
    if (rc) return rc;
    Control C;
    rc = read_control(c, &C);
    if (rc) return rc;
    if (out_host) fill_stats(C, out_host);
    return C.status;
}

int tga_descend_batch(tga_ctx **ctxs, int n, int64_t max_steps, tga_stats *out_host) {
    const Range range("tga_descend_batch");
    if (!ctxs || n < 0 || max_steps < 0) return TGA_ERR_INVALID;
    if (n == 0) return TGA_OK;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return TGA_ERR_INVALID;
        if (ctxs[i]->device != ctxs[0]->device) return TGA_ERR_INVALID;
        if (ctxs[i]->d.theta > 0) return TGA_ERR_STATE;      // the batched kernel has no edge-based path
        if (ctxs[i]->d.has_pd) return TGA_ERR_STATE;         // ... and no pickup path
    }
    int first = run_batch(ctxs, n, max_steps, 0, nullptr);
    for (int i = 0; i < n; ++i) {
        Control C;
        int rc = read_control(ctxs[i], &C);
        if (rc && !first) first = rc;
        if (!rc) {
            if (out_host) fill_stats(C, out_host + i);
            if (C.status && !first) first = C.status;
        }
    }
    return first;
}

int tga_batch_autotune(tga_ctx **ctxs, int n, int32_t *rows_out) {
    const Range range("tga_batch_autotune");
    if (!ctxs || n < 0) return TGA_ERR_INVALID;
    static const int bounds[] = {400, 800, 1400, 1 << 30};
    static const int trs[] = {16, 32, 64};
    int lo = 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TGA_ERR_CUDA;
    int rc = TGA_OK;
    for (int bi = 0; bi < 4 && !rc; ++bi) {
        std::vector<int> members;
        for (int i = 0; i < n; ++i)
            if (ctxs[i]->d.Wp >= lo && ctxs[i]->d.Wp < bounds[bi]) members.push_back(i);
        lo = bounds[bi];
        if (members.empty()) continue;
        std::sort(members.begin(), members.end(), [&](int a, int b) { return ctxs[a]->d.Wp < ctxs[b]->d.Wp; });
        tga_ctx *rep = ctxs[members[members.size() / 2]];
        int t16 = 16;
        rc = run_batch(&rep, 1, 1, 1, &t16);                // build once
        if (rc) break;
        float best = 1e30f;
        int best_tr = default_batch_tr(rep->d.Wp);
        for (int tr : trs) {
            cudaEventRecord(e0, rep->stream);
            for (int k = 0; k < 3 && !rc; ++k) rc = run_batch(&rep, 1, 1, 2, &tr);
            cudaEventRecord(e1, rep->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (!rc && ms < best) { best = ms; best_tr = tr; }
        }
        for (int i : members) ctxs[i]->batch_tr = best_tr;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rows_out)
        for (int i = 0; i < n; ++i) rows_out[i] = ctxs[i]->batch_tr ? ctxs[i]->batch_tr : default_batch_tr(ctxs[i]->d.Wp);
    // the tuning evaluations leave finished contexts behind: rebuild on next use
    for (int i = 0; i < n; ++i) ctxs[i]->built = false;
    return rc;
}

int tga_descend_async(tga_ctx *c, int64_t max_steps) {
    const Range range("tga_descend_async");
    if (!c || max_steps < 0) return TGA_ERR_INVALID;
    return descend_launch(c, max_steps);
}

int tga_query(tga_ctx *c, int32_t *done_out) {
    if (!c || !done_out) return TGA_ERR_INVALID;
    const cudaError_t e = cudaStreamQuery(c->stream);
    if (e == cudaSuccess) { *done_out = 1; return TGA_OK; }
    if (e == cudaErrorNotReady) { cudaGetLastError(); *done_out = 0; return TGA_OK; }
    return TGA_ERR_CUDA;
}

size_t tga_workspace_bytes(int32_t n_customers, int32_t n_routes) {
    if (n_customers < 1 || n_routes < 1) return 0;
    // the largest layout (pickup and swaps-of-runs records included): an upper bound
    return workspace_layout((size_t)n_customers, (size_t)n_routes, true, true).bytes;
}

int tga_sync(tga_ctx *c) {
    if (!c) return TGA_ERR_INVALID;
    Control C;
    int rc = read_control(c, &C);
    return rc ? rc : C.status;
}

int tga_get_stats(tga_ctx *c, tga_stats *out_host) {
    if (!c || !out_host) return TGA_ERR_INVALID;
    Control C;
    int rc = read_control(c, &C);
    if (rc) return rc;
    fill_stats(C, out_host);
    return TGA_OK;
}

int tga_get_op_candidates(tga_ctx *c, int64_t *out_host) {
    if (!c || !out_host) return TGA_ERR_INVALID;
    Control C;
    int rc = read_control(c, &C);
    if (rc) return rc;
    for (int op = 0; op < 8; ++op) out_host[op] = C.cand_op[op];
    return TGA_OK;
}

int tga_set_move_log(tga_ctx *c, uint64_t *log_dev, int64_t capacity) {
    if (!c || capacity < 0) return TGA_ERR_INVALID;
    c->d.log = (unsigned long long *)log_dev;
    c->d.log_cap = log_dev ? capacity : 0;
    drop_graph(c);
    return TGA_OK;
}

// Time `steps` steps of a descent from the saved solution along one path
// (persistent with the given shape, or the graph); milliseconds per
// evaluation, or a negative value if the path cannot run.
static float time_path(tga_ctx *c, int steps, bool persistent, int rows, int warps, int rs, cudaEvent_t e0,
                cudaEvent_t e1) {
    const size_t n = (size_t)c->d.n, m = (size_t)c->d.m;
    cudaMemcpyAsync(c->d.tour, c->saved, sizeof(int) * n, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->d.route_start, c->saved + n, sizeof(int) * (m + 1), cudaMemcpyDeviceToDevice, c->stream);
    if (tga_build_attrs(c) != TGA_OK) return -1.f;
    launch_begin(c->d, steps, c->stream);
    cudaEventRecord(e0, c->stream);
    int rc = TGA_OK;
    if (persistent) {
        int grid = 0;
        rc = persist_shape(rows, warps, rs, c->d, c->stream, &grid);
    } else {
        rc = build_graph(c);
        if (!rc && cudaGraphLaunch(c->gexec, c->stream) != cudaSuccess) rc = TGA_ERR_CUDA;
    }
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    Control C;
    if (rc || read_control(c, &C) || C.status || C.evals < 1) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / (float)C.evals;
}

// Measured choice of the automatic descent path: short descents from the
// current solution along the graph path (the tuned inter tile) and the
// persistent path under each block shape of 128 or 256 threads; the fastest
// per evaluation wins.  The caller's solution is restored and the
// attributes rebuilt afterwards.
static int tune_descent(tga_ctx *c, cudaEvent_t e0, cudaEvent_t e1) {
    // rows, column warps, row split (0: strip mode)
    static const int pshapes[][3] = {{8, 2, 2},  {16, 2, 2}, {16, 4, 1}, {16, 4, 2}, {16, 2, 4},
                                     {32, 2, 2}, {32, 4, 1}, {32, 4, 2}, {32, 8, 1}, {64, 4, 1},
                                     {64, 8, 1}, {16, 4, 0}, {16, 8, 0}, {32, 4, 0}, {32, 8, 0}};
    const int steps = 24;
    const size_t n = (size_t)c->d.n, m = (size_t)c->d.m;
    cudaMemcpyAsync(c->saved, c->d.tour, sizeof(int) * n, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->saved + n, c->d.route_start, sizeof(int) * (m + 1), cudaMemcpyDeviceToDevice, c->stream);
    unsigned long long *log = c->d.log;
    const long long cap = c->d.log_cap;
    c->d.log = nullptr;                                  // tuning descents are not recorded
    c->d.log_cap = 0;
    drop_graph(c);
    float best = time_path(c, steps, false, 0, 0, 0, e0, e1);
    int choice = best > 0.f ? TGA_DESCENT_GRAPH : 0;
    int br = 0, bw = 0, brs = 0;
    for (const auto &p : pshapes) {
        const float ms = time_path(c, steps, true, p[0], p[1], p[2], e0, e1);
        if (ms > 0.f && (choice == 0 || ms < best)) {
            best = ms;
            choice = TGA_DESCENT_PERSISTENT;
            br = p[0]; bw = p[1]; brs = p[2];
        }
    }
    cudaGetLastError();
    c->d.log = log;
    c->d.log_cap = cap;
    drop_graph(c);
    c->auto_choice = choice;
    c->ptile_rows = br; c->ptile_warps = bw; c->ptile_rs = brs;
    cudaMemcpyAsync(c->d.tour, c->saved, sizeof(int) * n, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->d.route_start, c->saved + n, sizeof(int) * (m + 1), cudaMemcpyDeviceToDevice, c->stream);
    return tga_build_attrs(c);
}

int tga_set_tile(tga_ctx *c, int32_t rows, int32_t warps) {
    const Range range("tga_set_tile");
    if (!c) return TGA_ERR_INVALID;
    if (rows != 0 || warps != 0) return set_tiles(c, rows, warps);
    if (!c->built) return TGA_ERR_STATE;
    // autotune: time every shape on the current state (evaluation only; the
    // solution is not touched), keep the fastest.
    // rows, column warps, row split, strip-major kernel
    static const int shapes[][4] = {{8, 2, 1, 0},  {16, 2, 1, 0}, {16, 2, 2, 0}, {16, 2, 4, 0}, {16, 4, 1, 0},
                                    {16, 4, 2, 0}, {32, 2, 2, 0}, {32, 2, 4, 0}, {32, 4, 1, 0}, {32, 4, 2, 0},
                                    {64, 4, 1, 0}, {64, 4, 2, 0}, {32, 8, 1, 0}, {64, 8, 1, 0}, {16, 4, 1, 1},
                                    {16, 8, 1, 1}, {32, 4, 1, 1}, {32, 8, 1, 1}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float bestms = 1e30f;
    int br = 32, bw = 4, brs = 1, bst = 0;
    for (const auto &s : shapes) {
        if (set_tiles(c, s[0], s[1], s[2], s[3] != 0) != TGA_OK) continue;
        launch_begin(c->d, 1, c->stream);
        launch_inter(c->d, c->tiles, c->ntiles, c->tile_rows, c->tile_warps, c->stream, c->tile_rs, 0, c->strip);
        cudaEventRecord(e0, c->stream);
        for (int k = 0; k < 5; ++k)
            launch_inter(c->d, c->tiles, c->ntiles, c->tile_rows, c->tile_warps, c->stream, c->tile_rs, 0,
                         c->strip);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < bestms) { bestms = ms; br = s[0]; bw = s[1]; brs = s[2]; bst = s[3]; }
    }
    // leave the context as it was before tuning (no pending key)
    cudaMemsetAsync(&c->d.ctl->best_key, 0xff, sizeof(unsigned long long), c->stream);
    int rc = set_tiles(c, br, bw, brs, bst != 0);
    if (!rc && c->mode == TGA_DESCENT_AUTO) rc = tune_descent(c, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    return check_launch();
}

int tga_set_descent_mode(tga_ctx *c, int32_t mode) {
    if (!c || mode < TGA_DESCENT_AUTO || mode > TGA_DESCENT_HOST) return TGA_ERR_INVALID;
    c->mode = mode;
    return TGA_OK;
}

int tga_get_descent_mode(tga_ctx *c, int32_t *last_used, int32_t *grid_out) {
    if (!c || !last_used) return TGA_ERR_INVALID;
    *last_used = c->last_mode;
    if (grid_out) *grid_out = c->last_mode == TGA_DESCENT_PERSISTENT ? c->persist_grid : 0;
    return TGA_OK;
}

int tga_set_persistent_shape(tga_ctx *c, int32_t rows, int32_t col_warps, int32_t row_split) {
    if (!c) return TGA_ERR_INVALID;
    if (rows == 0) {
        c->ptile_rows = c->ptile_warps = c->ptile_rs = 0;
        return TGA_OK;
    }
    const bool rows_ok = rows == 8 || rows == 16 || rows == 32 || rows == 64;
    const bool warps_ok = col_warps == 2 || col_warps == 4 || col_warps == 8;
    bool ok;
    if (row_split == 0) {
        ok = (rows == 16 || rows == 32) && (col_warps == 4 || col_warps == 8);
    } else {
        const int nt = col_warps * row_split * 32;
        ok = rows_ok && warps_ok && (row_split == 1 || row_split == 2 || row_split == 4) && (nt == 128 || nt == 256) &&
             rows % row_split == 0;
    }
    if (!ok) return TGA_ERR_INVALID;
    c->ptile_rows = rows; c->ptile_warps = col_warps; c->ptile_rs = row_split;
    return TGA_OK;
}

int tga_get_persistent_shape(tga_ctx *c, int32_t *rows, int32_t *col_warps, int32_t *row_split) {
    if (!c || !rows || !col_warps || !row_split) return TGA_ERR_INVALID;
    if (c->ptile_rows) {
        *rows = c->ptile_rows; *col_warps = c->ptile_warps; *row_split = c->ptile_rs;
        return TGA_OK;
    }
    if (!c->tiles && c->built && c->d.Wp > 2) default_tiles(c);
    int rs = c->tile_rs;
    while (c->tile_warps * 32 * rs < 128 && rs < 4 && c->tile_warps * rs * 2 <= 8 && c->tile_rows % (rs * 2) == 0)
        rs *= 2;
    *rows = c->tile_rows; *col_warps = c->tile_warps; *row_split = rs;
    return TGA_OK;
}

int tga_set_tile_shape(tga_ctx *c, int32_t rows, int32_t col_warps, int32_t row_split) {
    if (!c) return TGA_ERR_INVALID;
    return set_tiles(c, rows, col_warps, row_split);
}

int tga_get_tile_shape(tga_ctx *c, int32_t *rows, int32_t *col_warps, int32_t *row_split) {
    if (!c || !rows || !col_warps || !row_split) return TGA_ERR_INVALID;
    if (!c->tiles && c->built && c->d.Wp > 2) default_tiles(c);
    *rows = c->tile_rows;
    *col_warps = c->tile_warps;
    *row_split = c->strip ? 0 : c->tile_rs;
    return TGA_OK;
}

int tga_set_tile_strip(tga_ctx *c, int32_t rows, int32_t col_warps) {
    if (!c) return TGA_ERR_INVALID;
    return set_tiles(c, rows, col_warps, 1, true);
}

int tga_get_tile(tga_ctx *c, int32_t *rows, int32_t *warps) {
    if (!c || !rows || !warps) return TGA_ERR_INVALID;
    if (!c->tiles && c->built && c->d.Wp > 2) default_tiles(c);
    *rows = c->tile_rows;
    *warps = c->tile_warps;
    return TGA_OK;
}

int tga_profile_inter(tga_ctx *c, int32_t reps, float *ms_per_launch) {
    if (!c || reps < 1 || !ms_per_launch) return TGA_ERR_INVALID;
    if (!c->built) return TGA_ERR_STATE;
    if (!c->tiles && c->d.Wp > 2) default_tiles(c);
    return profile_launches(c, reps, ms_per_launch, [&] {
        launch_inter(c->d, c->tiles, c->ntiles, c->tile_rows, c->tile_warps, c->stream, c->tile_rs, 0, c->strip);
    });
}

int tga_profile_xswap(tga_ctx *c, int32_t reps, float *ms_per_launch) {
    if (!c || reps < 1 || !ms_per_launch) return TGA_ERR_INVALID;
    if (!c->built || !(c->d.op_mask & kExtOps)) return TGA_ERR_STATE;
    return profile_launches(c, reps, ms_per_launch, [&] { launch_xswap(c->d, c->stream); });
}

int tga_debug_read(tga_ctx *c, int32_t what, void *host_dst, size_t bytes, size_t *size_out) {
    if (!c) return TGA_ERR_INVALID;
    const Dev &d = c->d;
    const void *src = nullptr;
    size_t size = 0;
    switch (what) {
        case 0: src = d.ctl; size = sizeof(Control); break;
        case 1: src = d.seq; size = sizeof(int) * (size_t)d.Wp; break;
        case 2: src = d.pos_of; size = sizeof(int) * (size_t)(d.W + 1); break;
        case 3: src = d.brec; size = sizeof(BRec) * (size_t)(d.W + 1); break;
        case 4: src = d.erec; size = sizeof(ERec) * (size_t)(d.W + 1); break;
        case 5: src = d.rrec; size = sizeof(RouteRec) * (size_t)d.m; break;
        case 6: src = d.pcol; size = sizeof(int) * (size_t)(d.n + 1) * (size_t)d.ldp; break;
        case 7: src = c->tiles; size = sizeof(int2) * (size_t)c->ntiles; break;
        default: return TGA_ERR_INVALID;
    }
    if (size_out) *size_out = size;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return TGA_ERR_CUDA;
    if (host_dst && bytes && src) {
        if (cudaMemcpy(host_dst, src, bytes < size ? bytes : size, cudaMemcpyDeviceToHost) != cudaSuccess)
            return TGA_ERR_CUDA;
    }
    return TGA_OK;
}

int tga_get_bounds_report(tga_ctx *c, int64_t out[4]) {
    if (!c || !out) return TGA_ERR_INVALID;
    out[0] = out[1] = out[2] = out[3] = 0;
#ifdef TGA_BOUNDS_CHECK
    out[0] = 1;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return TGA_ERR_CUDA;
    Control h;
    if (cudaMemcpy(&h, c->d.ctl, sizeof(Control), cudaMemcpyDeviceToHost) != cudaSuccess) return TGA_ERR_CUDA;
    out[1] = h.bad_site;
    out[2] = h.bad_index;
    out[3] = h.bad_limit;
#endif
    return TGA_OK;
}

int tga_set_granular(tga_ctx *c, const int32_t *nbr_dev, int32_t theta) {
    if (!c || theta < 0) return TGA_ERR_INVALID;
    if (theta > 0 && (!nbr_dev || theta > c->d.n - 1)) return TGA_ERR_INVALID;
    if (theta > 0 && c->d.has_pd) return TGA_ERR_STATE;      // the edge-based kernel has no pickup path
    if (theta > 0 && (c->d.op_mask & kExtOps)) return TGA_ERR_STATE;   // ... and no swaps of runs
    if (c->granular) cudaFreeAsync(c->granular, c->stream);
    c->granular = nullptr;
    c->d.theta = 0; c->d.nbr = nullptr; c->d.nbr_rev = nullptr;
    drop_graph(c);
    c->auto_choice = 0;
    if (theta == 0) return check_launch();
    const size_t flags = align_up((size_t)(c->d.n + 1) * (size_t)theta, 256);
    if (cudaMallocAsync(&c->granular, flags + 256, c->stream) != cudaSuccess) {
        cudaGetLastError();
        c->granular = nullptr;
        return TGA_ERR_NOMEM;
    }
    unsigned char *rev = (unsigned char *)c->granular;
    int *bad = (int *)(rev + flags);
    Dev g = c->d;
    g.theta = theta; g.nbr = nbr_dev;
    int h_bad = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) { launch_granular_setup(g, rev, bad, c->stream); e = cudaGetLastError(); }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess || h_bad) {
        cudaFreeAsync(c->granular, c->stream);
        c->granular = nullptr;
        return e != cudaSuccess ? TGA_ERR_CUDA : TGA_ERR_INVALID;
    }
    c->d.theta = theta; c->d.nbr = nbr_dev; c->d.nbr_rev = rev;
    return TGA_OK;
}

int tga_set_wait_limit(tga_ctx *c, int64_t limit_ns) {
    if (!c) return TGA_ERR_INVALID;
    c->d.wait_ns = limit_ns < 0 ? -1 : (long long)limit_ns;
    drop_graph(c);                     // the captured launches carry the limit
    return TGA_OK;
}

int tga_destroy(tga_ctx *c) {
    if (!c) return TGA_ERR_INVALID;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->granular) cudaFreeAsync(c->granular, c->stream);
    c->granular = nullptr;
    drop_graph(c);
    if (c->tiles) cudaFreeAsync(c->tiles, c->stream);
    if (c->ws) cudaFreeAsync(c->ws, c->stream);
    if (c->tiles || c->ws) cudaStreamSynchronize(c->stream);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->cap2) cudaStreamDestroy(c->cap2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
    return TGA_OK;
}

}  // extern "C"
