// C ABI of the projector entry points (bsgd.h): forward and back projection
// over selected row / column blocks and the voxel-ray update count.
#include <algorithm>
#include <set>

#include "bsgd_internal.h"

namespace bsgd {
const char *last_error_cstr();
}

using namespace bsgd;

namespace {

bsgd_status block_lists(const bsgd_geometry *g, const int32_t *row_blocks, int n_rb,
                        const int32_t *col_blocks, int n_cb, std::vector<int> &rows,
                        std::vector<std::pair<int, int>> &runs) {
    rows.clear();
    runs.clear();
    BSGD_TRY(check_device(g));
    if (row_blocks) {
        if (n_rb < 1) return fail(BSGD_ERR_INVALID_ARG, "n_rb must be >= 1");
        std::set<int> seen;
        for (int k = 0; k < n_rb; ++k) {
            const int i = row_blocks[k];
            if (i < 0 || i >= g->M) return fail(BSGD_ERR_INVALID_ARG, "row block id out of range");
            if (!seen.insert(i).second) return fail(BSGD_ERR_INVALID_ARG, "duplicate row block id");
            rows.push_back(i);
        }
    } else {
        for (int i = 0; i < g->M; ++i) rows.push_back(i);
    }
    std::vector<int> cols;
    if (col_blocks) {
        if (n_cb < 1) return fail(BSGD_ERR_INVALID_ARG, "n_cb must be >= 1");
        for (int k = 0; k < n_cb; ++k) {
            const int j = col_blocks[k];
            if (j < 0 || j >= g->N) return fail(BSGD_ERR_INVALID_ARG, "column block id out of range");
            cols.push_back(j);
        }
        std::sort(cols.begin(), cols.end());
        if (std::adjacent_find(cols.begin(), cols.end()) != cols.end())
            return fail(BSGD_ERR_INVALID_ARG, "duplicate column block id");
    } else {
        for (int j = 0; j < g->N; ++j) cols.push_back(j);
    }
    // contiguous runs of column blocks share one traversal
    for (size_t k = 0; k < cols.size();) {
        size_t e = k + 1;
        while (e < cols.size() && cols[e] == cols[e - 1] + 1) ++e;
        runs.push_back({cols[k], cols[e - 1] + 1});
        k = e;
    }
    return BSGD_OK;
}

}  // namespace

extern "C" const char *bsgd_last_error(void) { return last_error_cstr(); }

extern "C" const char *bsgd_status_string(bsgd_status s) {
    switch (s) {
        case BSGD_OK: return "ok";
        case BSGD_ERR_INVALID_ARG: return "invalid argument";
        case BSGD_ERR_OOM: return "out of memory";
        case BSGD_ERR_CUDA: return "CUDA error";
        case BSGD_ERR_TIMEOUT: return "timeout";
        case BSGD_ERR_BUDGET: return "over budget";
        case BSGD_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

extern "C" bsgd_status bsgd_forward_project(const bsgd_geometry *g, const void *x, bsgd_dtype xt,
                                            void *y, bsgd_dtype yt, const int32_t *row_blocks,
                                            int n_rb, const int32_t *col_blocks, int n_cb,
                                            int accumulate, int batch, void *stream) {
    if (!g || !x || !y) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!dtype_ok(xt) || !dtype_ok(yt)) return fail(BSGD_ERR_INVALID_ARG, "bad dtype");
    if (batch < 1) return fail(BSGD_ERR_INVALID_ARG, "batch must be >= 1");
    std::vector<int> rows;
    std::vector<std::pair<int, int>> runs;
    BSGD_TRY(block_lists(g, row_blocks, n_rb, col_blocks, n_cb, rows, runs));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t C = g->n_cols(), R = g->n_rows();
    // y-fastest copy of each image for the views whose rays run along x; the
    // projection is the same without it (only slower), so a failed allocation
    // is not an error
    void *xT = nullptr;
    if (plain_wants_transpose(g, rows.data(), (int)rows.size()))
        pool_try_alloc(&xT, (size_t)C * dtype_size(xt), st);
    auto run_all = [&]() -> bsgd_status {
        for (int b = 0; b < batch; ++b) {
            const char *xb = (const char *)x + (size_t)b * C * dtype_size(xt);
            char *yb = (char *)y + (size_t)b * R * dtype_size(yt);
            if (!accumulate) BSGD_TRY(zero_rows(g, rows.data(), (int)rows.size(), yb, yt, st));
            for (auto &run : runs) {
                if (xT) BSGD_TRY(plain_transpose(g, xb, xt, xT, run.first, run.second, st));
                PlainLaunch L{rows.data(), (int)rows.size(), run.first, run.second, 0};
                BSGD_TRY(launch_fp_plain(g, L, xb, xt, yb, yt, 1, st, xT));
            }
        }
        return BSGD_OK;
    };
    const bsgd_status s = run_all();
    pool_free(xT, st);
    return s;
}

extern "C" bsgd_status bsgd_back_project(const bsgd_geometry *g, const void *r, bsgd_dtype rt,
                                         void *x, bsgd_dtype xt, const int32_t *row_blocks,
                                         int n_rb, const int32_t *col_blocks, int n_cb,
                                         float scale, int accumulate, int batch, void *stream) {
    if (!g || !x || !r) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!dtype_ok(rt)) return fail(BSGD_ERR_INVALID_ARG, "bad dtype");
    if (xt != BSGD_F32) return fail(BSGD_ERR_INVALID_ARG, "back projection writes float32 only");
    if (batch < 1) return fail(BSGD_ERR_INVALID_ARG, "batch must be >= 1");
    std::vector<int> rows;
    std::vector<std::pair<int, int>> runs;
    BSGD_TRY(block_lists(g, row_blocks, n_rb, col_blocks, n_cb, rows, runs));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t C = g->n_cols(), R = g->n_rows();
    // y-fastest FP32 accumulator for the views whose rays run along x, added
    // back into x after each run (optional, as in the forward projection)
    float *gT = nullptr;
    if (plain_wants_transpose(g, rows.data(), (int)rows.size()))
        pool_try_alloc((void **)&gT, (size_t)C * 4, st);
    auto run_all = [&]() -> bsgd_status {
        for (int b = 0; b < batch; ++b) {
            const char *rb = (const char *)r + (size_t)b * R * dtype_size(rt);
            float *xb = (float *)x + (size_t)b * C;
            for (auto &run : runs) {
                const int64_t v0 = (int64_t)g->plane_start[run.first] * g->dg.plane_stride;
                const int64_t v1 = (int64_t)g->plane_start[run.second] * g->dg.plane_stride;
                if (!accumulate) BSGD_CUDA(cudaMemsetAsync(xb + v0, 0, (v1 - v0) * 4, st));
                if (gT) BSGD_CUDA(cudaMemsetAsync(gT + v0, 0, (v1 - v0) * 4, st));
                PlainLaunch L{rows.data(), (int)rows.size(), run.first, run.second, 0};
                BSGD_TRY(launch_bp_plain(g, L, rb, rt, xb, scale, st, gT));
                if (gT) BSGD_TRY(plain_add_transposed(g, gT, xb, run.first, run.second, st));
            }
        }
        return BSGD_OK;
    };
    const bsgd_status s = run_all();
    pool_free(gT, st);
    return s;
}

extern "C" bsgd_status bsgd_count_updates(const bsgd_geometry *g, const int32_t *row_blocks,
                                          int n_rb, const int32_t *col_blocks, int n_cb,
                                          int64_t *out, void *stream) {
    if (!g || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    std::vector<int> rows;
    std::vector<std::pair<int, int>> runs;
    BSGD_TRY(block_lists(g, row_blocks, n_rb, col_blocks, n_cb, rows, runs));
    cudaStream_t st = (cudaStream_t)stream;
    const int V = g->desc.n_views;
    unsigned long long *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 8 * (size_t)V);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BSGD_ERR_OOM, "cudaMalloc of the counters failed");
    }
    auto run = [&]() -> bsgd_status {
        BSGD_CUDA(cudaMemsetAsync(d, 0, 8 * (size_t)V, st));
        for (auto &r : runs) {
            PlainLaunch L{rows.data(), (int)rows.size(), r.first, r.second, 0};
            BSGD_TRY(launch_count(g, L, d, st));
        }
        std::vector<unsigned long long> h(V);
        BSGD_CUDA(cudaMemcpyAsync(h.data(), d, 8 * (size_t)V, cudaMemcpyDeviceToHost, st));
        BSGD_CUDA(cudaStreamSynchronize(st));
        int64_t tot = 0;
        for (auto c : h) tot += (int64_t)c;
        *out = tot;
        return BSGD_OK;
    };
    bsgd_status s = run();
    cudaFree(d);
    return s;
}
