// TV proximal step of BSGD-TV (Algorithm 4): x <- argmin_t ||t - x||^2 +
// 2 kappa TV(t), kappa = mu * lambda, with the isotropic TV of Eq. 10 built from
// backward differences (a difference with no neighbour is zero; 3D volumes use
// all three axes). The paper leaves the inner solver open; this is FGP (Beck
// and Teboulle 2009): projected gradient with momentum on the dual field p,
// |p(c)| <= 1, t = b - kappa D^T p, step 1 / (kappa L), L = 4 * ndim.
//
// Per iteration two stencil passes over the volume, both HBM-bound:
//   tv_primal_kernel  u = b - kappa D^T r          (reads r at c and c + e_k)
//   tv_dual_kernel    p = P(r + D u / (kappa L)),  r = p + w (p - p_prev)
// Threads are laid out 32 x 8 over (x, y) of one z plane, so voxel coordinates
// come from the launch indices and neighbours along x share cache lines. The
// dual fields are one float4 per voxel: with a separate array per component
// the dual pass ran at 6 % of HBM bandwidth (six read-modify-write streams
// whose accesses fell on the same memory channels), with float4 it streams.
#include <algorithm>
#include <cmath>

#include "siddon_device.cuh"

namespace bsgd {

struct TvDims {
    int nx, ny, nz, ndim;
    int64_t n;
};

__device__ __forceinline__ bool tv_voxel(const TvDims &D, int &x, int &y, int &z, int64_t &k) {
    x = blockIdx.x * 32 + (threadIdx.x & 31);
    y = blockIdx.y * 8 + (threadIdx.x >> 5);
    z = blockIdx.z;
    k = ((int64_t)z * D.ny + y) * D.nx + x;
    return x < D.nx && y < D.ny;
}

// u = b - kappa D^T r; D^T r at c = sum_k r_k[c] [c_k >= 1] - r_k[c + e_k] [c_k <= n_k - 2].
// The dual fields are stored one float4 per voxel (x, y, z components, one
// unused): one 16-byte access per voxel instead of a stream per component.
// With ulo (16-bit image with its low-order term) u is split into u + ulo.
template <typename TO>
__global__ void __launch_bounds__(256) tv_primal_kernel(const TvDims D, const float *__restrict__ b,
                                                        const float4 *__restrict__ r, float kappa,
                                                        TO *__restrict__ u,
                                                        TO *__restrict__ ulo = nullptr) {
    int x, y, z;
    int64_t k;
    if (!tv_voxel(D, x, y, z, k)) return;
    const int64_t sy = D.nx, sz = (int64_t)D.nx * D.ny;
    const float4 rc = r[k];
    float dt = 0.f;
    if (x >= 1) dt += rc.x;
    if (x <= D.nx - 2) dt -= r[k + 1].x;
    if (y >= 1) dt += rc.y;
    if (y <= D.ny - 2) dt -= r[k + sy].y;
    if (D.ndim == 3) {
        if (z >= 1) dt += rc.z;
        if (z <= D.nz - 2) dt -= r[k + sz].z;
    }
    const float val = b[k] - kappa * dt;
    if (ulo == nullptr) {
        stf(u + k, val);
    } else {
        const float hi = rnd(val, u);
        stf(u + k, hi);
        stf(ulo + k, val - hi);
    }
}

template <typename T>
__global__ void add_lo_kernel(float *__restrict__ b, const T *__restrict__ lo, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        b[k] += ldv(lo + k);
}

__global__ void __launch_bounds__(256) tv_dual_kernel(const TvDims D, const float *__restrict__ u,
                                                      float step, float wgt, float4 *__restrict__ r,
                                                      float4 *__restrict__ p_prev) {
    int x, y, z;
    int64_t k;
    if (!tv_voxel(D, x, y, z, k)) return;
    const int64_t sy = D.nx, sz = (int64_t)D.nx * D.ny;
    const float uc = u[k];
    const float4 rc = r[k], po = p_prev[k];
    const float q0 = rc.x + step * (x >= 1 ? uc - u[k - 1] : 0.f);
    const float q1 = rc.y + step * (y >= 1 ? uc - u[k - sy] : 0.f);
    const float q2 = D.ndim == 3 ? rc.z + step * (z >= 1 ? uc - u[k - sz] : 0.f) : 0.f;
    const float nrm = sqrtf(fmaf(q0, q0, fmaf(q1, q1, q2 * q2)));
    const float sc = 1.0f / fmaxf(1.0f, nrm);
    const float p0 = q0 * sc, p1 = q1 * sc, p2 = q2 * sc;
    p_prev[k] = make_float4(p0, p1, p2, 0.f);
    r[k] = make_float4(fmaf(wgt, p0 - po.x, p0), fmaf(wgt, p1 - po.y, p1), fmaf(wgt, p2 - po.z, p2), 0.f);
}

bsgd_status convert(const void *in, bsgd_dtype it, void *out, bsgd_dtype ot, int64_t n,
                    cudaStream_t st);

static TvDims tv_dims(const bsgd_geometry *g) {
    return TvDims{g->desc.nx, g->desc.ny, g->desc.nz, g->desc.nz > 1 ? 3 : 2, g->n_cols()};
}

bsgd_status tv_work_alloc(const bsgd_geometry *g, TvWork &w) {
    const TvDims D = tv_dims(g);
    const size_t n = (size_t)D.n;
    cudaError_t e1 = cudaMalloc(&w.b, n * 4), e2 = cudaMalloc(&w.u, n * 4),
                e3 = cudaMalloc(&w.p, n * 16), e4 = cudaMalloc(&w.r, n * 16);
    if (e1 || e2 || e3 || e4) {
        cudaGetLastError();
        cudaFree(w.b), cudaFree(w.u), cudaFree(w.p), cudaFree(w.r);
        w = TvWork{};
        return fail(BSGD_ERR_OOM, "TV prox: cannot allocate the dual field");
    }
    return BSGD_OK;
}

void tv_work_free(TvWork &w) {
    cudaFree(w.b);
    cudaFree(w.u);
    cudaFree(w.p);
    cudaFree(w.r);
    w = TvWork{};
}

// The prox on stream st with a caller-owned workspace: launches only, no host
// synchronisation.
bsgd_status tv_prox_run(const bsgd_geometry *g, void *x, bsgd_dtype xt, double kappa, int iters,
                        cudaStream_t st, void *xlo, const TvWork &w) {
    if (!(kappa > 0) || iters < 1) return BSGD_OK;
    const TvDims D = tv_dims(g);
    const int64_t n = D.n;
    BSGD_TRY(convert(x, xt, w.b, BSGD_F32, n, st));
    const int gb0 = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
    if (xlo && xt == BSGD_BF16) add_lo_kernel<<<gb0, 256, 0, st>>>(w.b, (const __nv_bfloat16 *)xlo, n);
    if (xlo && xt == BSGD_F16) add_lo_kernel<<<gb0, 256, 0, st>>>(w.b, (const __half *)xlo, n);
    BSGD_CUDA(cudaMemsetAsync(w.p, 0, (size_t)n * 16, st));
    BSGD_CUDA(cudaMemsetAsync(w.r, 0, (size_t)n * 16, st));
    const dim3 grid((D.nx + 31) / 32, (D.ny + 7) / 8, D.nz);
    const float L = 4.0f * D.ndim;
    const float step = (float)(1.0 / (kappa * L));
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        tv_primal_kernel<float><<<grid, 256, 0, st>>>(D, w.b, w.r, (float)kappa, w.u);
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        tv_dual_kernel<<<grid, 256, 0, st>>>(D, w.u, step, (float)((t - 1.0) / tn), w.r, w.p);
        t = tn;
    }
    if (xt == BSGD_F32)
        tv_primal_kernel<float><<<grid, 256, 0, st>>>(D, w.b, w.p, (float)kappa, (float *)x);
    else if (xt == BSGD_BF16)
        tv_primal_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(D, w.b, w.p, (float)kappa,
                                                              (__nv_bfloat16 *)x, (__nv_bfloat16 *)xlo);
    else
        tv_primal_kernel<__half><<<grid, 256, 0, st>>>(D, w.b, w.p, (float)kappa, (__half *)x,
                                                       (__half *)xlo);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

}  // namespace bsgd

extern "C" bsgd_status bsgd_tv_prox(const bsgd_geometry *g, void *x, bsgd_dtype xt, double kappa,
                                    int iters, void *stream) {
    using namespace bsgd;
    if (!g || !x) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!dtype_ok(xt)) return fail(BSGD_ERR_INVALID_ARG, "bad dtype");
    if (!(kappa >= 0) || iters < 0) return fail(BSGD_ERR_INVALID_ARG, "kappa >= 0, iters >= 0");
    if (g->desc.nz > 65535) return fail(BSGD_ERR_INVALID_ARG, "TV prox supports nz <= 65535");
    BSGD_TRY(check_device(g));
    if (!(kappa > 0) || iters < 1) return BSGD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    TvWork w;
    BSGD_TRY(tv_work_alloc(g, w));
    bsgd_status s = tv_prox_run(g, x, xt, kappa, iters, st, nullptr, w);
    if (cudaStreamSynchronize(st) != cudaSuccess && !s) s = fail(BSGD_ERR_CUDA, "TV prox failed");
    tv_work_free(w);
    return s;
}
