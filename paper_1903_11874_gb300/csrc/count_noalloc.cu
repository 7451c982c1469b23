// Voxel-ray update count that allocates no memory.
//
// bsgd_count_updates keeps one counter per view in device memory it allocates
// for the call. Some callers cannot let a library allocate device memory: a
// process whose device memory is owned by a caching allocator or reserved up
// front by a framework, a serving loop that must not block on cudaMalloc /
// cudaFree (both can synchronise the device), or code that runs where the
// allocator is off limits. For them this variant keeps its counters in a
// file-scope __device__ array of fixed size instead.
//
// Limits and sharing: the array holds kNoAllocMaxViews counters plus one total,
// so geometries with more views are rejected. Every GPU that loads this library
// holds the array (about 128 KiB) until the process exits. All calls on a
// device share it and it keeps the last call's contents: each call clears the
// counters first, and calls that overlap on the GPU (different streams, or
// host threads racing) corrupt each other's counts.
#include <mutex>

#include "siddon_device.cuh"

namespace bsgd {

constexpr int kNoAllocMaxViews = 16384;

// counters [0, kNoAllocMaxViews) per view, [kNoAllocMaxViews] the total
static __device__ __align__(256) unsigned long long g_noalloc_counts[kNoAllocMaxViews + 1];

namespace {

struct NoAllocRows {
    int n;
    int ids[64];
};

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned long long *g_addr[kMaxDevices] = {};

// Device address of the counters on the current device. The host-side name
// g_noalloc_counts is only a stand-in for the symbol, so kernels must be given
// this address. Looked up once per device (the first call on a device does it).
bsgd_status counter_address(unsigned long long **out) {
    int dev = 0;
    BSGD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(BSGD_ERR_INVALID_ARG, "device id out of range");
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_counts);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_counts)");
        g_addr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_addr[dev];
    return BSGD_OK;
}

__device__ __forceinline__ int noalloc_view(const DeviceGeom &G, const NoAllocRows &R, int slot) {
    const int k = slot / G.max_views, pos = slot % G.max_views;
    if (k >= R.n) return -1;
    const int i = R.ids[k];
    return pos < G.block_nviews[i] ? G.block_views[i * G.max_views + pos] : -1;
}

// Same traversal and threshold as the update count of bsgd_count_updates.
template <bool k3D>
__global__ void __launch_bounds__(128) count_noalloc_kernel(const DeviceGeom G, const NoAllocRows R,
                                                            int j0, int j1,
                                                            unsigned long long *counts) {
    const int a = noalloc_view(G, R, blockIdx.y);
    if (a < 0) return;
    const Band b = band_of(G, a, j0, j1);
    int u, v, nt;
    if (!tile_pixel<k3D>(b, blockIdx.x, u, v, nt)) return;
    RayWalk w;
    unsigned long long c = 0;
    if (ray_setup(G, a, u, v, G.plane_start[j0], G.plane_start[j1], w)) {
        const float eps = 1e-4f * fminf(G.hx, fminf(G.hy, G.hz)) / w.L;
        ray_walk(w, [&](int, float s) { c += s > eps ? 1ull : 0ull; });
    }
    if (c) atomicAdd(counts + a, c);
}

__global__ void total_noalloc_kernel(unsigned long long *counts, int n) {
    unsigned long long acc = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += counts[k];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ unsigned long long part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
        counts[kNoAllocMaxViews] = t;
    }
}

}  // namespace
}  // namespace bsgd

using namespace bsgd;

extern "C" bsgd_status bsgd_count_updates_noalloc(const bsgd_geometry *g, const int32_t *row_blocks,
                                                  int n_rb, const int32_t *col_blocks, int n_cb,
                                                  int64_t *out, void *stream) {
    if (!g || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    const int V = g->desc.n_views;
    if (V > kNoAllocMaxViews)
        return fail(BSGD_ERR_INVALID_ARG,
                    "bsgd_count_updates_noalloc supports at most 16384 views (its counters are a "
                    "fixed array); use bsgd_count_updates");
    if (g->N > kNoAllocMaxViews) return fail(BSGD_ERR_INVALID_ARG, "too many column blocks");
    // the kernels run on the current device: it must be the one holding the
    // geometry's tables
    BSGD_TRY(check_device(g));
    // selected blocks as bit sets on the stack (4 KiB in all: this entry point
    // allocates nothing, on the device or on the host)
    constexpr int kWords = kNoAllocMaxViews / 32;
    uint32_t seen_r[kWords] = {}, cols[kWords] = {};
    auto has = [](const uint32_t *set, int k) { return (set[k >> 5] >> (k & 31)) & 1u; };
    auto put = [](uint32_t *set, int k) { set[k >> 5] |= 1u << (k & 31); };
    int nr = g->M;
    if (row_blocks) {
        if (n_rb < 1) return fail(BSGD_ERR_INVALID_ARG, "n_rb must be >= 1");
        for (int k = 0; k < n_rb; ++k) {
            const int i = row_blocks[k];
            if (i < 0 || i >= g->M) return fail(BSGD_ERR_INVALID_ARG, "row block id out of range");
            if (has(seen_r, i)) return fail(BSGD_ERR_INVALID_ARG, "duplicate row block id");
            put(seen_r, i);
        }
        nr = n_rb;
    }
    if (col_blocks) {
        if (n_cb < 1) return fail(BSGD_ERR_INVALID_ARG, "n_cb must be >= 1");
        for (int k = 0; k < n_cb; ++k) {
            const int j = col_blocks[k];
            if (j < 0 || j >= g->N) return fail(BSGD_ERR_INVALID_ARG, "column block id out of range");
            if (has(cols, j)) return fail(BSGD_ERR_INVALID_ARG, "duplicate column block id");
            put(cols, j);
        }
    } else {
        for (int j = 0; j < g->N; ++j) put(cols, j);
    }
    unsigned long long *counts = nullptr;
    BSGD_TRY(counter_address(&counts));
    cudaStream_t st = (cudaStream_t)stream;
    BSGD_CUDA(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (kNoAllocMaxViews + 1), st));
    const bool t3 = g->desc.nv > 1;
    const int tu = tile_u(g), tv = tile_v(g);
    for (int j0 = 0; j0 < g->N;) {
        if (!has(cols, j0)) { ++j0; continue; }
        int j1 = j0 + 1;
        while (j1 < g->N && has(cols, j1)) ++j1;
        for (int k0 = 0; k0 < nr; k0 += 64) {
            NoAllocRows R{};
            R.n = nr - k0 < 64 ? nr - k0 : 64;
            int tiles = 0;
            for (int k = 0; k < R.n; ++k) {
                R.ids[k] = row_blocks ? row_blocks[k0 + k] : k0 + k;
                for (int a : g->block_views[R.ids[k]]) {
                    Band b{1 << 30, -1, 1 << 30, -1};
                    if (j0 == 0 && j1 == g->N) {
                        b = g->bands[(size_t)a * (g->N + 1) + g->N];
                    } else {
                        for (int j = j0; j < j1; ++j) {
                            const Band &c = g->bands[(size_t)a * (g->N + 1) + j];
                            if (c.u0 > c.u1 || c.v0 > c.v1) continue;
                            b.u0 = b.u0 < c.u0 ? b.u0 : c.u0;
                            b.u1 = b.u1 > c.u1 ? b.u1 : c.u1;
                            b.v0 = b.v0 < c.v0 ? b.v0 : c.v0;
                            b.v1 = b.v1 > c.v1 ? b.v1 : c.v1;
                        }
                    }
                    if (b.u0 > b.u1 || b.v0 > b.v1) continue;
                    const int t = ((b.u1 - b.u0 + tu) / tu) * ((b.v1 - b.v0 + tv) / tv);
                    tiles = t > tiles ? t : tiles;
                }
            }
            if (tiles == 0) continue;
            dim3 grid(tiles, R.n * g->max_views);
            if (t3) count_noalloc_kernel<true><<<grid, 128, 0, st>>>(g->dg, R, j0, j1, counts);
            else count_noalloc_kernel<false><<<grid, 128, 0, st>>>(g->dg, R, j0, j1, counts);
            BSGD_CUDA(cudaGetLastError());
        }
        j0 = j1;
    }
    total_noalloc_kernel<<<1, 256, 0, st>>>(counts, V);
    BSGD_CUDA(cudaGetLastError());
    unsigned long long total = 0;
    BSGD_CUDA(cudaMemcpyAsync(&total, counts + kNoAllocMaxViews, sizeof(total),
                              cudaMemcpyDeviceToHost, st));
    BSGD_CUDA(cudaStreamSynchronize(st));
    *out = (int64_t)total;
    return BSGD_OK;
}
