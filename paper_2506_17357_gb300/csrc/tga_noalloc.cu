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

namespace tga {
namespace {

constexpr int kNoAllocMaxPositions = 1280;     // n + m + 1
constexpr int kNoAllocRows = 16, kNoAllocWarps = 4;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

constexpr size_t ldp_for(size_t positions) {
    return (positions + kMaxTileCols - 1) / kMaxTileCols * kMaxTileCols + 16;
}

constexpr size_t tiles_upper_bound(size_t positions) {
    const size_t TC = kNoAllocWarps * 32;
    return ((positions + kNoAllocRows - 1) / kNoAllocRows) * ((positions + TC - 1) / TC);
}

// Scratch layout for n customers, m routes: the arrays of a context plus
// the tile list.  Returns the bytes; fills d's pointers when base != null.
size_t noalloc_layout(Dev &d, int2 **tiles, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t n = (size_t)d.n, m = (size_t)d.m, W = (size_t)d.W, P = (size_t)d.Wp;
    const size_t o_ctl = take(sizeof(Control));
    const size_t o_seq = take(sizeof(int) * P);
    const size_t o_pos = take(sizeof(int) * (W + 1));
    const size_t o_brec = take(sizeof(BRec) * (W + 1));
    const size_t o_erec = take(sizeof(ERec) * (W + 1));
    const size_t o_prec = take(sizeof(PRec) * (W + 1));
    const size_t o_xrec = take(sizeof(XRec) * (W + 1));
    const size_t o_rrec = take(sizeof(RouteRec) * m);
    const size_t o_seen = take(sizeof(int) * (n + 1));
    const size_t o_intra = take(sizeof(int) * kIntraVecPD * (P + m));
    const size_t o_tiles = take(sizeof(int2) * tiles_upper_bound(P));
    const size_t o_pcol = take(sizeof(int) * (n + 1) * (size_t)d.ldp);
    if (base) {
        d.ctl = (Control *)(base + o_ctl);
        d.seq = (int *)(base + o_seq);
        d.pos_of = (int *)(base + o_pos);
        d.brec = (BRec *)(base + o_brec);
        d.erec = (ERec *)(base + o_erec);
        d.prec = (PRec *)(base + o_prec);
        d.xrec = (XRec *)(base + o_xrec);
        d.rrec = (RouteRec *)(base + o_rrec);
        d.seen = (int *)(base + o_seen);
        d.scr_intra = (int *)(base + o_intra);
        d.pcol = (int *)(base + o_pcol);
        *tiles = (int2 *)(base + o_tiles);
    }
    return off;
}

// Bytes at the largest admitted sizes, each piece bounded independently
// (n+1 <= 1280, m <= 1279, W+1 <= 1281, positions <= 1280).
constexpr size_t noalloc_max_bytes() {
    const size_t P = kNoAllocMaxPositions, N1 = P, M = P - 1, W1 = P + 1;
    return align256(sizeof(Control)) + align256(4 * P) + align256(4 * W1) + align256(sizeof(BRec) * W1) +
           align256(sizeof(ERec) * W1) + align256(sizeof(PRec) * W1) + align256(sizeof(XRec) * W1) +
           align256(sizeof(RouteRec) * M) +
           align256(4 * N1) + align256(4 * kIntraVecPD * (P + M)) +
           align256(sizeof(int2) * tiles_upper_bound(P)) + align256(4 * N1 * ldp_for(P));
}

constexpr size_t kNoAllocBytes = noalloc_max_bytes();

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
    // tiles of row tiles 0..I-1 precede row tile I; row tile J0 is the first
    // column tile with a pair p < q
    long long before = 0;
    for (int k = 0; k < I; ++k) {
        const long long j0 = ((long long)k * rows + 1 + cols - 1) / cols - 1;   // first J with (J+1)*cols-1 > k*rows
        const long long jj = j0 < 0 ? 0 : j0;
        before += nct > jj ? nct - jj : 0;
    }
    long long j0 = ((long long)I * rows + 1 + cols - 1) / cols - 1;
    if (j0 < 0) j0 = 0;
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
    d.ldp = (int)ldp_for((size_t)d.Wp);
    d.log = nullptr; d.log_cap = 0;

    int2 *tiles = nullptr;
    if (noalloc_layout(d, &tiles, nullptr) > kNoAllocBytes) return TGA_ERR_RANGE;
    char *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    noalloc_layout(d, &tiles, base);
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
    if (cudaStreamSynchronize(s) != cudaSuccess) return TGA_ERR_CUDA;
    int status = 0;
    if (cudaMemcpy(&status, &d.ctl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TGA_ERR_CUDA;
    return status;
}
