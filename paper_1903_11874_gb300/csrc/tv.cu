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
#include <algorithm>
#include <cmath>

#include "siddon_device.cuh"

namespace bsgd {

struct TvDims {
    int nx, ny, nz, ndim;
    int64_t n;
};

__device__ __forceinline__ void tv_coords(const TvDims &D, int64_t k, int &x, int &y, int &z) {
    x = (int)(k % D.nx);
    y = (int)((k / D.nx) % D.ny);
    z = (int)(k / ((int64_t)D.nx * D.ny));
}

// u = b - kappa D^T r; D^T r at c = sum_k r_k[c] [c_k >= 1] - r_k[c + e_k] [c_k <= n_k - 2].
// With ulo (16-bit image with its low-order term) u is split into u + ulo.
template <typename TO>
__global__ void tv_primal_kernel(const TvDims D, const float *__restrict__ b,
                                 const float *__restrict__ r, float kappa, TO *__restrict__ u,
                                 TO *__restrict__ ulo = nullptr) {
    const int64_t sx = 1, sy = D.nx, sz = (int64_t)D.nx * D.ny;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < D.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        tv_coords(D, k, x, y, z);
        const float *rx = r, *ry = r + D.n, *rz = r + 2 * D.n;
        float dt = 0.f;
        if (x >= 1) dt += rx[k];
        if (x <= D.nx - 2) dt -= rx[k + sx];
        if (y >= 1) dt += ry[k];
        if (y <= D.ny - 2) dt -= ry[k + sy];
        if (D.ndim == 3) {
            if (z >= 1) dt += rz[k];
            if (z <= D.nz - 2) dt -= rz[k + sz];
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
}

template <typename T>
__global__ void add_lo_kernel(float *__restrict__ b, const T *__restrict__ lo, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        b[k] += ldv(lo + k);
}

__global__ void tv_dual_kernel(const TvDims D, const float *__restrict__ u, float step, float wgt,
                               float *__restrict__ r, float *__restrict__ p_prev) {
    const int64_t sx = 1, sy = D.nx, sz = (int64_t)D.nx * D.ny;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < D.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        tv_coords(D, k, x, y, z);
        const float uc = u[k];
        float q[3];
        q[0] = r[k] + step * (x >= 1 ? uc - u[k - sx] : 0.f);
        q[1] = r[D.n + k] + step * (y >= 1 ? uc - u[k - sy] : 0.f);
        q[2] = D.ndim == 3 ? r[2 * D.n + k] + step * (z >= 1 ? uc - u[k - sz] : 0.f) : 0.f;
        const float nrm = sqrtf(fmaf(q[0], q[0], fmaf(q[1], q[1], q[2] * q[2])));
        const float sc = 1.0f / fmaxf(1.0f, nrm);
        for (int a = 0; a < D.ndim; ++a) {
            const float pn = q[a] * sc;
            const float po = p_prev[a * D.n + k];
            p_prev[a * D.n + k] = pn;
            r[a * D.n + k] = fmaf(wgt, pn - po, pn);
        }
    }
}

bsgd_status convert(const void *in, bsgd_dtype it, void *out, bsgd_dtype ot, int64_t n,
                    cudaStream_t st);

bsgd_status tv_prox_impl(const bsgd_geometry *g, void *x, bsgd_dtype xt, double kappa, int iters,
                         cudaStream_t st, void *xlo) {
    if (!(kappa > 0) || iters < 1) return BSGD_OK;
    TvDims D{g->desc.nx, g->desc.ny, g->desc.nz, g->desc.nz > 1 ? 3 : 2, g->n_cols()};
    const int64_t n = D.n;
    float *b = nullptr, *u = nullptr, *p = nullptr, *r = nullptr;
    auto cleanup = [&]() { cudaFree(b); cudaFree(u); cudaFree(p); cudaFree(r); };
    cudaError_t e1 = cudaMalloc(&b, n * 4), e2 = cudaMalloc(&u, n * 4),
                e3 = cudaMalloc(&p, (size_t)D.ndim * n * 4), e4 = cudaMalloc(&r, (size_t)D.ndim * n * 4);
    if (e1 || e2 || e3 || e4) {
        cudaGetLastError();
        cleanup();
        return fail(BSGD_ERR_OOM, "TV prox: cannot allocate the dual field");
    }
    auto run = [&]() -> bsgd_status {
        BSGD_TRY(convert(x, xt, b, BSGD_F32, n, st));
        const int gb0 = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
        if (xlo && xt == BSGD_BF16) add_lo_kernel<<<gb0, 256, 0, st>>>(b, (const __nv_bfloat16 *)xlo, n);
        if (xlo && xt == BSGD_F16) add_lo_kernel<<<gb0, 256, 0, st>>>(b, (const __half *)xlo, n);
        BSGD_CUDA(cudaMemsetAsync(p, 0, (size_t)D.ndim * n * 4, st));
        BSGD_CUDA(cudaMemsetAsync(r, 0, (size_t)D.ndim * n * 4, st));
        const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
        const float L = 4.0f * D.ndim;
        const float step = (float)(1.0 / (kappa * L));
        double t = 1.0;
        for (int k = 0; k < iters; ++k) {
            tv_primal_kernel<float><<<gb, 256, 0, st>>>(D, b, r, (float)kappa, u);
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            tv_dual_kernel<<<gb, 256, 0, st>>>(D, u, step, (float)((t - 1.0) / tn), r, p);
            t = tn;
        }
        if (xt == BSGD_F32) tv_primal_kernel<float><<<gb, 256, 0, st>>>(D, b, p, (float)kappa, (float *)x);
        else if (xt == BSGD_BF16) tv_primal_kernel<__nv_bfloat16><<<gb, 256, 0, st>>>(D, b, p, (float)kappa, (__nv_bfloat16 *)x, (__nv_bfloat16 *)xlo);
        else tv_primal_kernel<__half><<<gb, 256, 0, st>>>(D, b, p, (float)kappa, (__half *)x, (__half *)xlo);
        BSGD_CUDA(cudaGetLastError());
        BSGD_CUDA(cudaStreamSynchronize(st));
        return BSGD_OK;
    };
    bsgd_status s = run();
    cleanup();
    return s;
}

}  // namespace bsgd

extern "C" bsgd_status bsgd_tv_prox(const bsgd_geometry *g, void *x, bsgd_dtype xt, double kappa,
                                    int iters, void *stream) {
    if (!g || !x) return bsgd::fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!bsgd::dtype_ok(xt)) return bsgd::fail(BSGD_ERR_INVALID_ARG, "bad dtype");
    if (!(kappa >= 0) || iters < 0) return bsgd::fail(BSGD_ERR_INVALID_ARG, "kappa >= 0, iters >= 0");
    return bsgd::tv_prox_impl(g, x, xt, kappa, iters, (cudaStream_t)stream, nullptr);
}
