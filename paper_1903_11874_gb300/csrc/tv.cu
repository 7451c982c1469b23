// TV proximal step of BSGD-TV (Algorithm 4): x <- argmin_t ||t - x||^2 +
// 2 kappa TV(t), kappa = mu * lambda, with the isotropic TV of Eq. 10 built from
// backward differences (a difference with no neighbour is zero; 3D volumes use
// all three axes). The paper leaves the inner solver open; this is FGP (Beck
// and Teboulle 2009): projected gradient with momentum on the dual field p,
// |p(c)| <= 1, t = b - kappa D^T p, step 1 / (kappa L), L = 4 * ndim.
//
// One iteration is one HBM-bound stencil pass (tv_fgp_kernel):
//   u = b - kappa D^T r            (r at c and c + e_k; u is never stored)
//   p = P(r + D u / (kappa L)),    r = p + w (p - p_prev)
// and the final image is one pass of tv_primal_kernel with r = p. The dual
// fields are one float4 per voxel: with a separate array per component the
// dual pass ran at 6 % of HBM bandwidth (six read-modify-write streams whose
// accesses fell on the same memory channels), with float4 it streams.
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

// Asynchronous global -> shared copies (cp.async): `bytes` from src, or zeros
// when `valid` is false (src must still be a mapped address; nothing is read).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One FGP iteration in one pass. A CTA of 256 threads owns a 32 x 8 (x, y)
// column of the volume over the planes [zb, zb + zchunk) and marches up in z.
// Plane z's stage holds the extrapolated dual r of the column with one voxel
// of halo on every side in x and y (34 x 10) and b on the 33 x 9 points whose
// u the plane's backward differences need (the column and its low-x / low-y
// neighbours); stages are filled by cp.async kTvAhead planes ahead in a ring
// of kTvAhead + 2. Per plane: u = b - kappa D^T r on the 33 x 9 points (r of this plane
// and of the next), then the dual of the CTA's own 32 x 8 voxels; u of the
// plane below is kept from the previous step (a CTA first computes u of the
// plane below its chunk). r is read from r_in and written to r_out: other CTAs
// still read r_in's halo. u is formed as tv_primal_kernel forms it, the dual
// step in the same order of operations as before the fusion.
constexpr int kTvTx = 32, kTvTy = 8;
constexpr int kTvRx = kTvTx + 2, kTvRy = kTvTy + 2;   // staged r region
constexpr int kTvUx = kTvTx + 1, kTvUy = kTvTy + 1;   // u points
constexpr int kTvAhead = 2;                   // planes staged ahead of the one in use
constexpr int kTvStages = kTvAhead + 2;       // + the plane in use and the one read two steps ago

struct TvStage {
    float4 r[kTvRy][kTvRx];
    float b[kTvUy][kTvUx];
};

__global__ void __launch_bounds__(256) tv_fgp_kernel(const TvDims D, const float *__restrict__ b,
                                                     const float4 *__restrict__ r_in, float kappa,
                                                     float step, float wgt, int zchunk,
                                                     float4 *__restrict__ r_out,
                                                     float4 *__restrict__ p_prev) {
    __shared__ TvStage stg[kTvStages];
    __shared__ float su[kTvUy][kTvUx];
    const int x0 = blockIdx.x * kTvTx, y0 = blockIdx.y * kTvTy;
    const int zb = blockIdx.z * zchunk, ze = min(D.nz, zb + zchunk);
    if (zb >= ze) return;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const bool three = D.ndim == 3;
    const int zs = three ? max(zb - 1, 0) : zb;
    // the last plane any step reads: the chunk's top plane's upper neighbour
    const int zlast = three ? min(ze, D.nz - 1) : ze - 1;
    auto stage_plane = [&](int z) {   // plane z into stage (z - zs) % kTvStages
        TvStage &S = stg[(z - zs) % kTvStages];
        for (int q = tid; q < kTvRx * kTvRy; q += 256) {
            const int lx = q % kTvRx, ly = q / kTvRx;
            const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            const bool ok = gx >= 0 && gx < D.nx && gy >= 0 && gy < D.ny;
            cp_async16(&S.r[ly][lx], ok ? r_in + ((int64_t)z * D.ny + gy) * D.nx + gx : r_in, ok);
        }
        for (int q = tid; q < kTvUx * kTvUy; q += 256) {
            const int lx = q % kTvUx, ly = q / kTvUx;
            const int ux = x0 - 1 + lx, uy = y0 - 1 + ly;
            const bool ok = ux >= 0 && ux < D.nx && uy >= 0 && uy < D.ny;
            cp_async4(&S.b[ly][lx], ok ? b + ((int64_t)z * D.ny + uy) * D.nx + ux : b, ok);
        }
    };
    for (int a = 0; a < kTvAhead; ++a) {
        if (zs + a <= zlast) stage_plane(zs + a);
        cp_async_commit();
    }
    float u_below = 0.f;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool mine = gx < D.nx && gy < D.ny;
    for (int z = zs; z < ze; ++z) {
        // kTvAhead planes ahead: its stage last held plane z - 2, read two steps ago
        if (z + kTvAhead <= zlast) stage_plane(z + kTvAhead);
        cp_async_commit();
        const int64_t k = ((int64_t)z * D.ny + gy) * D.nx + gx;
        float4 po = make_float4(0.f, 0.f, 0.f, 0.f);
        if (z >= zb && mine) po = p_prev[k];
        cp_async_wait<kTvAhead - 1>();   // planes z and z + 1 have landed (this thread's copies)
        __syncthreads();      // ... and every thread's
        const TvStage &C = stg[(z - zs) % kTvStages];
        const TvStage &Nx = stg[(z + 1 - zs) % kTvStages];
        for (int q = tid; q < kTvUx * kTvUy; q += 256) {
            const int lx = q % kTvUx, ly = q / kTvUx;
            const int ux = x0 - 1 + lx, uy = y0 - 1 + ly;
            float val = 0.f;
            if (ux >= 0 && ux < D.nx && uy >= 0 && uy < D.ny) {
                const float4 rc = C.r[ly][lx];
                float dt = 0.f;
                if (ux >= 1) dt += rc.x;
                if (ux <= D.nx - 2) dt -= C.r[ly][lx + 1].x;
                if (uy >= 1) dt += rc.y;
                if (uy <= D.ny - 2) dt -= C.r[ly + 1][lx].y;
                if (three) {
                    if (z >= 1) dt += rc.z;
                    if (z <= D.nz - 2) dt -= Nx.r[ly][lx].z;
                }
                val = C.b[ly][lx] - kappa * dt;
            }
            su[ly][lx] = val;
        }
        __syncthreads();
        const float uc = su[ty + 1][tx + 1];
        if (z >= zb && mine) {
            const float4 rc = C.r[ty + 1][tx + 1];
            const float q0 = rc.x + step * (gx >= 1 ? uc - su[ty + 1][tx] : 0.f);
            const float q1 = rc.y + step * (gy >= 1 ? uc - su[ty][tx + 1] : 0.f);
            const float q2 = three ? rc.z + step * (z >= 1 ? uc - u_below : 0.f) : 0.f;
            const float nrm = sqrtf(fmaf(q0, q0, fmaf(q1, q1, q2 * q2)));
            const float sc = 1.0f / fmaxf(1.0f, nrm);
            const float p0 = q0 * sc, p1 = q1 * sc, p2 = q2 * sc;
            p_prev[k] = make_float4(p0, p1, p2, 0.f);
            r_out[k] = make_float4(fmaf(wgt, p0 - po.x, p0), fmaf(wgt, p1 - po.y, p1),
                                   fmaf(wgt, p2 - po.z, p2), 0.f);
        }
        u_below = uc;
    }
    cp_async_wait<0>();
}

bsgd_status convert(const void *in, bsgd_dtype it, void *out, bsgd_dtype ot, int64_t n,
                    cudaStream_t st);

static TvDims tv_dims(const bsgd_geometry *g) {
    return TvDims{g->desc.nx, g->desc.ny, g->desc.nz, g->desc.nz > 1 ? 3 : 2, g->n_cols()};
}

bsgd_status tv_work_alloc(const bsgd_geometry *g, TvWork &w) {
    const TvDims D = tv_dims(g);
    const size_t n = (size_t)D.n;
    cudaError_t e1 = cudaMalloc(&w.b, n * 4), e2 = cudaMalloc(&w.r2, n * 16),
                e3 = cudaMalloc(&w.p, n * 16), e4 = cudaMalloc(&w.r, n * 16);
    if (e1 || e2 || e3 || e4) {
        cudaGetLastError();
        cudaFree(w.b), cudaFree(w.r2), cudaFree(w.p), cudaFree(w.r);
        w = TvWork{};
        return fail(BSGD_ERR_OOM, "TV prox: cannot allocate the dual field");
    }
    return BSGD_OK;
}

void tv_work_free(TvWork &w) {
    cudaFree(w.b);
    cudaFree(w.r2);
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
    // z-chunks per column: as many as keep every CTA resident in one wave
    // (the staging ring's shared memory sets the CTAs per SM), at least 8
    // planes a chunk
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        BSGD_CUDA(cudaGetDevice(&dev));
        BSGD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        BSGD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tv_fgp_kernel, 256, 0));
        resident = std::max(1, sms * per_sm);
    }
    const int64_t cols = (int64_t)grid.x * grid.y;
    const int max_chunks = std::max(1, D.nz / 8);
    const int chunks = (int)std::min<int64_t>(max_chunks, std::max<int64_t>(1, resident / cols));
    const int zchunk = (D.nz + chunks - 1) / chunks;
    const dim3 fgrid(grid.x, grid.y, (D.nz + zchunk - 1) / zchunk);
    float4 *rin = w.r, *rout = w.r2;
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        tv_fgp_kernel<<<fgrid, 256, 0, st>>>(D, w.b, rin, (float)kappa, step, (float)((t - 1.0) / tn),
                                             zchunk, rout, w.p);
        std::swap(rin, rout);
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
