// apd_cell_moments_noalloc: the per-cell moments of apd_cell_moments without a
// workspace, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a device-memory
// budget fixed when the process starts, code embedded in a host framework whose
// own allocator owns all device memory and rejects allocations made behind its
// back, or latency-critical loops where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable.  This entry point needs no allocation:
// its scratch (seed records, the near-tie queue and the device counters) lives
// in one file-scope __device__ array of fixed size, which every GPU that loads
// the library holds until the process exits.
//
// Limits: at most kMaxSeeds seeds and kMaxPixels pixels per call (about
// 8.5 MiB of static device memory).  All calls share the one array per device,
// so calls that overlap on the GPU (different streams, or host threads without
// ordering) race on it; the array keeps the last call's contents, and every
// call clears the parts that must start at zero.
#include <mutex>

#include "apd_internal.cuh"

namespace {

constexpr int kMaxSeeds = 4096;                  // multiple of the 256-seed chunk
constexpr long long kMaxPixels = 1ll << 21;      // 2,097,152 pixels
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    apd::SeedRec recs[kMaxSeeds];
    apd::SeedRec32 recs32[kMaxSeeds];
    uint32_t flags[kMaxPixels];
    apd::DevScalars sc;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_scratch_mu;
NoAllocScratch *g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device.  In host code
// the symbol is only a host-side stand-in, so the address is asked from the
// runtime once per device (with that device current) and cached.
int scratch_for_current_device(NoAllocScratch **out, int *device) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return APD_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return APD_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_scratch_addr[dev];
    *device = dev;
    return APD_OK;
}

int grid_of(const apd_grid *gr, apd::GridDev &g) {
    if (!gr || (gr->dim != 2 && gr->dim != 3)) return APD_ERR_ARG;
    g = apd::GridDev{};
    g.dim = gr->dim;
    long long J = 1;
    double cell = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (d < gr->dim) {
            if (gr->res[d] < 1 || !(gr->hi[d] > gr->lo[d]) || !isfinite(gr->lo[d]) || !isfinite(gr->hi[d]))
                return APD_ERR_ARG;
            g.res[d] = gr->res[d];
            g.lo[d] = gr->lo[d];
            g.h[d] = (gr->hi[d] - gr->lo[d]) / (double)gr->res[d];
            g.h32[d] = (float)g.h[d];
            J *= gr->res[d];
            cell *= g.h[d];
            if (J > kMaxPixels) return APD_ERR_WORKSPACE;
        } else {
            g.res[d] = 1;
            g.h[d] = 1.0;
            g.h32[d] = 1.f;
        }
    }
    g.J = J;
    g.cell = cell;
    return APD_OK;
}

int status_of(int bits) {
    if (bits & apd::ST_NOT_SPD) return APD_ERR_NOT_SPD;
    if (bits & (apd::ST_NONFINITE | apd::ST_BAD_VOLUME)) return APD_ERR_ARG;
    if (bits & apd::ST_TIMEOUT) return APD_ERR_TIMEOUT;
    if (bits) return APD_ERR_CUDA;
    return APD_OK;
}

}  // namespace

extern "C" int apd_cell_moments_noalloc(const apd_grid *grid, const apd_seeds *seeds, int64_t *moments,
                                        apd_stream_t stream) {
    apd::GridDev g;
    int rc = grid_of(grid, g);
    if (rc != APD_OK) return rc;
    if (!seeds || seeds->n < 1 || !seeds->x || !seeds->A || !seeds->w || !moments) return APD_ERR_ARG;
    if (seeds->n > kMaxSeeds) return APD_ERR_WORKSPACE;
    NoAllocScratch *s = nullptr;
    int dev = 0;
    rc = scratch_for_current_device(&s, &dev);
    if (rc != APD_OK) return rc;

    // a workspace view over the static scratch (no allocation)
    apd::Workspace ws;
    ws.dim = g.dim;
    ws.max_n = kMaxSeeds;
    ws.max_j = kMaxPixels;
    ws.device = dev;
    ws.n_pad_max = kMaxSeeds;
    ws.recs = s->recs;
    ws.recs32 = s->recs32;
    ws.flags = s->flags;
    ws.sc = &s->sc;

    const int n = seeds->n;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *mom = reinterpret_cast<unsigned long long *>(moments);
    const size_t K = (size_t)apd::moment_width(g.dim);
    // the counters, statistics and status word start at zero on every call
    if (cudaMemsetAsync(&s->sc, 0, sizeof(apd::DevScalars), st) != cudaSuccess) return APD_ERR_CUDA;
    if (cudaMemsetAsync(mom, 0, (size_t)n * K * sizeof(unsigned long long), st) != cudaSuccess)
        return APD_ERR_CUDA;
    if (apd::launch_eval_reset(ws, st) != cudaSuccess) return APD_ERR_CUDA;
    if (apd::launch_seed_prep(g, n, seeds->x, seeds->A, seeds->w, ws, st) != cudaSuccess) return APD_ERR_CUDA;
    if (apd::launch_assign_fp32(g, n, ws, nullptr, mom, st) != cudaSuccess) return APD_ERR_CUDA;
    if (apd::launch_rescore_fp64(g, n, seeds->x, seeds->A, seeds->w, ws, nullptr, mom, st) != cudaSuccess)
        return APD_ERR_CUDA;
    // device-side checks (non-finite input, A not SPD, a wait that timed out)
    int bits = 0;
    if (cudaMemcpyAsync(&bits, &s->sc.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return APD_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return APD_ERR_CUDA;
    return status_of(bits);
}
