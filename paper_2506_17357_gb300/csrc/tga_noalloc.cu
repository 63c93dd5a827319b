// Allocation-free best-move evaluation.
//
// Some callers cannot allocate device memory at all: code that runs inside
// another framework's memory pool with the CUDA allocator locked down,
// plugins that are handed a stream and pre-allocated buffers only, or hosts
// that forbid cudaMalloc after start-up so memory use stays fixed.
// tga_eval_best_move_noalloc serves them: it evaluates the neighbourhood of
// a caller-supplied instance + solution and writes the best move, using as
// its only scratch a file-scope device array of fixed size.  Nothing is
// allocated -- no cudaMalloc, no cudaFree, no allocating library routine.
//
// The array is part of the library image: every GPU that loads libtga holds
// it (kNoAllocBytes) until the process exits.  In host code its name is only
// a host-side stand-in, so its device address is looked up once per device
// with cudaGetSymbolAddress (on the first call for that device, with that
// device current) and passed to the kernels as a plain pointer.  The kernels
// are the same ones the context path runs; only where their scratch lives
// differs.
#include <mutex>

#include "tga_internal.cuh"
#undef TGA_FILE_ID
#define TGA_FILE_ID 6

namespace tga {
namespace {

constexpr int kNoAllocMaxPositions = 1280;     // n + m + 1
constexpr int kNoAllocRows = 16, kNoAllocWarps = 4;

constexpr size_t tiles_upper_bound(size_t positions) {
    const size_t TC = kNoAllocWarps * 32;
    return ((positions + kNoAllocRows - 1) / kNoAllocRows) * ((positions + TC - 1) / TC);
}

// Scratch bytes for n customers and m routes: the workspace of a context
// (the same layout, with the pickup and swaps-of-runs records) followed by
// the inter-route tile list.
constexpr size_t noalloc_bytes(const WsLayout &L, size_t positions) {
    return L.bytes + ws_align(sizeof(int2) * tiles_upper_bound(positions));
}

// The array's size: the layout at the largest admitted sizes, each bounded
// on its own (n+1 <= 1280 nodes, m <= 1279 routes, W+1 <= 1281 anchor
// records, 1280 positions).  The layout grows with each of them, so this
// bounds the scratch of every admitted instance.
constexpr size_t kNoAllocBytes =
    noalloc_bytes(workspace_pieces(kNoAllocMaxPositions, kNoAllocMaxPositions - 1, kNoAllocMaxPositions + 1,
                                   kNoAllocMaxPositions, true, true),
                  kNoAllocMaxPositions);
static_assert(kNoAllocBytes < (size_t)8 << 20, "the allocation-free scratch stays below 8 MB");

// Point d's arrays (and *tiles) into the scratch at base.
void noalloc_carve(Dev &d, int2 **tiles, char *base) {
    const WsLayout L = workspace_layout((size_t)d.n, (size_t)d.m, true, true);
    d.ctl = (Control *)(base + L.ctl);
    d.seq = (int *)(base + L.seq);
    d.pos_of = (int *)(base + L.pos);
    d.brec = (BRec *)(base + L.brec);
    d.erec = (ERec *)(base + L.erec);
    d.prec = (PRec *)(base + L.prec);
    d.xrec = (XRec *)(base + L.xrec);
    d.rrec = (RouteRec *)(base + L.rrec);
    d.seen = (int *)(base + L.seen);
    d.scr_intra = (int *)(base + L.intra);
    d.pcol = (int *)(base + L.pcol);
    *tiles = (int2 *)(base + L.bytes);
}

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char *g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TGA_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TGA_ERR_CUDA;
        }
        g_scratch_ptr[dev] = (char *)p;
    }
    *out = g_scratch_ptr[dev];
    return TGA_OK;
}

// Upper-triangle tile list of the inter-route evaluation, written on the
// device (one thread per row tile) so the host never stages it.
__global__ void k_noalloc_tiles(int2 *tiles, int nrt, int nct, int rows, int cols) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nrt) return;
    // tiles of row tiles 0..I-1 precede row tile I; in row tile k the first
    // column tile holding a pair p < q is the first J with
    // (J+1)*cols - 1 > k*rows, i.e. J = floor((k*rows + 1) / cols)
    long long before = 0;
    for (int k = 0; k < I; ++k) {
        const long long j0 = ((long long)k * rows + 1) / cols;
        before += nct > j0 ? nct - j0 : 0;
    }
    const long long j0 = ((long long)I * rows + 1) / cols;
    for (long long J = j0; J < nct; ++J) tiles[before + (J - j0)] = make_int2(I, (int)J);
}

}  // namespace
}  // namespace tga

using namespace tga;

extern "C" int tga_eval_best_move_noalloc(const tga_instance *inst, const tga_solution *sol,
                                          uint32_t op_mask, tga_stream_t stream, tga_move *out_dev) {
    if (!inst || !sol || !out_dev) return TGA_ERR_INVALID;
    const long long n = inst->n_customers, m = inst->n_routes;
    if (n < 1 || m < 1 || inst->capacity < 0 || inst->w_load < 0 || inst->w_tw < 0) return TGA_ERR_INVALID;
    if (op_mask == 0 || op_mask >= 256u) return TGA_ERR_INVALID;
    if (!inst->dist || !inst->demand || !sol->tour || !sol->route_start) return TGA_ERR_INVALID;
    if (inst->has_tw && (!inst->service || !inst->tw_early || !inst->tw_late)) return TGA_ERR_INVALID;
    if (inst->pickup && !inst->has_tw) return TGA_ERR_INVALID;
    if (inst->pickup && (op_mask & kExtOps)) return TGA_ERR_INVALID;
    if (n + m + 1 > kNoAllocMaxPositions) return TGA_ERR_RANGE;

    Dev d{};
    d.n = (int)n; d.m = (int)m; d.W = (int)(n + 1 + m); d.Wp = (int)(n + m + 1);
    d.Q = inst->capacity; d.wL = inst->w_load; d.wT = inst->w_tw; d.has_tw = inst->has_tw ? 1 : 0;
    d.op_mask = op_mask;
    d.dist = inst->dist; d.demand = inst->demand;
    d.service = inst->service; d.early = inst->tw_early; d.late = inst->tw_late;
    d.has_pd = inst->pickup ? 1 : 0;
    d.pickup = inst->pickup;
    d.tour = sol->tour; d.route_start = sol->route_start;
    d.cvrp_by_route = cvrp_intra_by_route(d.n, d.m, d.has_tw, d.op_mask);
    d.ldp = (int)pcol_pitch((size_t)d.Wp);
    d.log = nullptr; d.log_cap = 0;
    d.wait_ns = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || d.nsm < 1) {
        cudaGetLastError();
        return TGA_ERR_CUDA;
    }

    int2 *tiles = nullptr;
    if (noalloc_bytes(workspace_layout((size_t)n, (size_t)m, true, true), (size_t)d.Wp) > kNoAllocBytes)
        return TGA_ERR_RANGE;
    char *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    noalloc_carve(d, &tiles, base);
    if (setup_kernel_attrs(d.Wp) != 0) return TGA_ERR_CUDA;

    const int Wa = d.Wp - 1, TC = kNoAllocWarps * 32;
    const int nrt = (Wa + kNoAllocRows - 1) / kNoAllocRows, nct = (Wa + TC - 1) / TC;
    long long ntiles = 0;
    for (int I = 0; I < nrt; ++I)
        for (int J = 0; J < nct; ++J)
            if ((long long)(J + 1) * TC - 1 > (long long)I * kNoAllocRows) ++ntiles;

    cudaStream_t s = (cudaStream_t)stream;
    // the control block is the only state that must start from zero; every
    // other array is fully written before it is read
    if (cudaMemsetAsync(d.ctl, 0, sizeof(Control), s) != cudaSuccess) return TGA_ERR_CUDA;
    k_noalloc_tiles<<<(nrt + 127) / 128, 128, 0, s>>>(tiles, nrt, nct, kNoAllocRows, TC);
    launch_check_instance(d, s);
    launch_build(d, s);
    launch_begin(d, 1, s);
    launch_eval(d, tiles, (int)ntiles, kNoAllocRows, kNoAllocWarps, s);
    launch_finalize(d, out_dev, s);
    if (cudaGetLastError() != cudaSuccess) return TGA_ERR_CUDA;
    // the status word is read on the caller's stream only, so work queued on
    // other streams is not waited for
    int status = 0;
    if (cudaMemcpyAsync(&status, &d.ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return TGA_ERR_CUDA;
    return status;
}
