// Siddon projector kernels: plain FP / BP / segment count over selected blocks,
// and the two solver kernels of one BSGD iteration (FP with the fused residual
// update, BP of the residual change).
//
// Grid of the plain BP and count kernels and the solver's BP: x = tile of the
// detector band (128 rays per CTA), y = view slot inside the selected row
// block(s), z = pair slot (solver). FP and fused kernels: x = tile x view slots
// with the view slot fastest (z = pair slot in the solver). A CTA's rays all belong to one view and one
// column block, so they share the view's ray table entry and walk a compact
// bundle of neighbouring voxels.
#include <algorithm>
#include <type_traits>

#include "siddon_device.cuh"

namespace bsgd {

// Selected row blocks of a plain launch (views = block_views of each).
struct RowSel {
    int n;
    int ids[64];
};

__device__ __forceinline__ int sel_view(const DeviceGeom &G, const RowSel &R, int slot) {
    const int k = slot / G.max_views, pos = slot % G.max_views;
    if (k >= R.n) return -1;
    const int i = R.ids[k];
    return pos < G.block_nviews[i] ? G.block_views[i * G.max_views + pos] : -1;
}

// ---------------------------------------------------------------------------
// Plain kernels

// Views whose rays run along x gather from xT (y fastest) when it is given, so
// that the lanes of a warp (neighbouring detector columns) read neighbouring
// addresses; the other views read x.
template <bool k3D, typename TX, typename TY>
__global__ void __launch_bounds__(128) fp_plain_kernel(const DeviceGeom G, const RowSel R, int j0,
                                                       int j1, const TX *__restrict__ x,
                                                       TY *__restrict__ y,
                                                       const TX *__restrict__ xT) {
    // view slot fastest (as in the solver's FP): the CTAs running together
    // gather the same band rows of every view
    const int a = sel_view(G, R, blockIdx.x % (R.n * G.max_views));
    if (a < 0) return;
    const Band b = band_of(G, a, j0, j1);
    int u, v, nt;
    if (!tile_pixel<k3D>(b, blockIdx.x / (R.n * G.max_views), u, v, nt)) return;
    const bool yf = xT != nullptr && G.view_yfast[a];
    const TX *src = yf ? xT : x;
    RayWalk w;
    float acc = 0.f;
    if (ray_setup(G, a, u, v, G.plane_start[j0], G.plane_start[j1], w, yf)) {
        ray_walk_fast(w, [&](int idx, float s) { acc = fmaf(s, ldf(src + idx), acc); });
        acc *= w.L;
    }
    const int64_t row = ((int64_t)a * G.nv + v) * G.nu + u;
    stf(y + row, ldv(y + row) + acc);
}

// Views whose rays run along x scatter into gT (y fastest) when it is given.
template <bool k3D, typename TR>
__global__ void __launch_bounds__(128) bp_plain_kernel(const DeviceGeom G, const RowSel R, int j0,
                                                       int j1, const TR *__restrict__ r,
                                                       float *__restrict__ x, float scale,
                                                       float *__restrict__ gT) {
    const int a = sel_view(G, R, blockIdx.y);
    if (a < 0) return;
    const Band b = band_of(G, a, j0, j1);
    int u, v, nt;
    if (!tile_pixel<k3D>(b, blockIdx.x, u, v, nt)) return;
    const int64_t row = ((int64_t)a * G.nv + v) * G.nu + u;
    const float rv = ldf(r + row) * scale;
    if (rv == 0.f) return;
    const bool yf = gT != nullptr && G.view_yfast[a];
    float *dst = yf ? gT : x;
    RayWalk w;
    if (!ray_setup(G, a, u, v, G.plane_start[j0], G.plane_start[j1], w, yf)) return;
    const float wl = rv * w.L;
    ray_walk_fast(w, [&](int idx, float s) {
        if (s > 0.f) atomicAdd(dst + idx, s * wl);
    });
}

// out[z][x][y] = in[z][y][x] for the planes z0 <= z < z1, through a 32 x 33
// shared tile so that both the reads and the writes are coalesced.
template <typename T>
__global__ void __launch_bounds__(256) transpose_planes_kernel(const DeviceGeom G, int z0, int z1,
                                                               const T *__restrict__ in,
                                                               T *__restrict__ out) {
    __shared__ float sx[32][33];
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int tx_n = (G.nx + 31) / 32, ty_n = (G.ny + 31) / 32;
    const int64_t ntiles = (int64_t)tx_n * ty_n * (z1 - z0);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int z = z0 + (int)(t / (tx_n * ty_n)), rem = (int)(t % (tx_n * ty_n));
        const int x0 = (rem % tx_n) * 32, y0 = (rem / tx_n) * 32;
        __syncthreads();
        for (int k = row; k < 32; k += 8) {
            const int yy = y0 + k, xx = x0 + lane;
            if (xx < G.nx && yy < G.ny) sx[k][lane] = ldf(in + ((int64_t)z * G.ny + yy) * G.nx + xx);
        }
        __syncthreads();
        for (int k = row; k < 32; k += 8) {
            const int xx = x0 + k, yy = y0 + lane;
            if (xx < G.nx && yy < G.ny) stf(out + ((int64_t)z * G.nx + xx) * G.ny + yy, sx[lane][k]);
        }
    }
}

// x[z][y][x] += gT[z][x][y] for the planes z0 <= z < z1.
__global__ void __launch_bounds__(256) add_transposed_kernel(const DeviceGeom G, int z0, int z1,
                                                             const float *__restrict__ gT,
                                                             float *__restrict__ x) {
    __shared__ float sg[32][33];
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int tx_n = (G.nx + 31) / 32, ty_n = (G.ny + 31) / 32;
    const int64_t ntiles = (int64_t)tx_n * ty_n * (z1 - z0);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int z = z0 + (int)(t / (tx_n * ty_n)), rem = (int)(t % (tx_n * ty_n));
        const int x0 = (rem % tx_n) * 32, y0 = (rem / tx_n) * 32;
        __syncthreads();
        for (int k = row; k < 32; k += 8) {           // gT rows: fixed x, consecutive y
            const int xx = x0 + k, yy = y0 + lane;
            if (xx < G.nx && yy < G.ny) sg[k][lane] = gT[((int64_t)z * G.nx + xx) * G.ny + yy];
        }
        __syncthreads();
        for (int k = row; k < 32; k += 8) {           // x rows: fixed y, consecutive x
            const int yy = y0 + k, xx = x0 + lane;
            if (xx < G.nx && yy < G.ny) x[((int64_t)z * G.ny + yy) * G.nx + xx] += sg[lane][k];
        }
    }
}

// Voxel-ray updates (segments longer than 1e-4 of the smallest voxel edge;
// shorter pieces are edge / corner crossings, zero in exact arithmetic),
// accumulated per (view, cell) into counts.
template <bool k3D>
__global__ void __launch_bounds__(128) count_kernel(const DeviceGeom G, const RowSel R, int j0,
                                                    int j1, int n_cells,
                                                    unsigned long long *__restrict__ counts) {
    const int a = sel_view(G, R, blockIdx.y);
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
    if (c == 0) return;
    int cell = 0;
    if (n_cells == 2) cell = u >= G.nu / 2;
    if (n_cells == 4) cell = (v >= G.nv / 2) * 2 + (u >= G.nu / 2);
    atomicAdd(counts + (size_t)a * n_cells + cell, c);
}

__global__ void zero_views_kernel(const DeviceGeom G, const RowSel R, void *y, int esize) {
    const int a = sel_view(G, R, blockIdx.y);
    if (a < 0) return;
    const int64_t per = (int64_t)G.nv * G.nu;
    char *base = reinterpret_cast<char *>(y) + (size_t)a * per * esize;
    const int64_t nbytes = per * esize;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; k < nbytes;
         k += (int64_t)gridDim.x * blockDim.x * 4) {
        if (k + 4 <= nbytes && ((reinterpret_cast<uintptr_t>(base + k) & 3) == 0))
            *reinterpret_cast<uint32_t *>(base + k) = 0u;
        else
            for (int t = 0; t < 4 && k + t < nbytes; ++t) base[k + t] = 0;
    }
}

// ---------------------------------------------------------------------------
// Solver kernels

__device__ __forceinline__ bool solve_pixel(const DeviceGeom &G, const SolveDev &S, int tile,
                                            int slot, int p, int &a, int &i, int &j, int &u,
                                            int &v, bool &in_band) {
    const Work &W = *S.work;
    if (p >= W.n_pairs) return false;
    i = W.pair_i[p];
    j = W.pair_j[p];
    if (slot >= G.block_nviews[i]) return false;
    a = G.block_views[i * G.max_views + slot];
    Band b = G.bands[(size_t)a * (G.N + 1) + j];
    if (S.n_cells > 1) cell_rect(G.nu, G.nv, S.n_cells, S.cells[p * G.max_views + slot], b);
    int nt;
    in_band = G.nv > 1 ? tile_pixel<true>(b, tile, u, v, nt) : tile_pixel<false>(b, tile, u, v, nt);
    return tile < nt;
}

// FP of the pair's rows for one CTA work item (detector tile, view slot, pair):
// z_new = A_R^J x_J; with FUSED also z^J = z_new, r = y - sum_j z^j and the FP64
// row-block residual sums S. The early returns are uniform over the CTA.
template <typename T, bool FUSED>
__device__ __forceinline__ void fp_solve_body(const DeviceGeom &G, const SolveDev &S,
                                              const T *__restrict__ x, int tile, int slot, int p) {
    int a, i, j, u, v;
    bool act;
    if (!solve_pixel(G, S, tile, slot, p, a, i, j, u, v, act)) return;
    if (S.owned && !S.owned[j]) return;   // another process owns block j
    float zn = 0.f;
    if (act) {
        const bool yf = S.xT != nullptr && G.view_yfast[a];
        const T *src = yf ? reinterpret_cast<const T *>(S.xT) : x;
        RayWalk w;
        if (ray_setup(G, a, u, v, G.plane_start[j], G.plane_start[j + 1], w, yf)) {
            float acc = 0.f;
            ray_walk_fast(w, [&](int idx, float s) { acc = fmaf(s, ldf(src + idx), acc); });
            zn = acc * w.L;
        }
    }
    const int64_t row = act ? ((int64_t)a * G.nv + v) * G.nu + u : 0;
    T *z = reinterpret_cast<T *>(S.z);
    bool in;
    if (!FUSED) {
        if (act) stf(z + zslot(G, j, a, u, v, in), zn);
        return;
    }
    double dn = 0.0;
    if (act) {
        stf(z + zslot(G, j, a, u, v, in), zn);
        zn = rnd(zn, z);
        float zs = 0.f;
        for (int jj = 0; jj < G.N; ++jj) {   // z^jj is 0 outside block jj's band
            if (jj == j) {
                zs += zn;
                continue;
            }
            const int64_t k = zslot(G, jj, a, u, v, in);
            if (in) zs += ldv(z + k);
        }
        T *r = reinterpret_cast<T *>(S.r);
        const float rn = rnd(ldf(reinterpret_cast<const T *>(S.y) + row) - zs, r);
        const float ro = ldv(r + row);
        stf(r + row, rn);
        dn = (double)rn * rn - (double)ro * ro;
    }
    // the 32 lanes of a warp share one detector row; lane 0 has the lowest u,
    // so it is active whenever any lane of the warp is
    for (int o = 16; o > 0; o >>= 1) dn += __shfl_xor_sync(0xffffffffu, dn, o);
    if ((threadIdx.x & 31) == 0 && act && dn != 0.0) atomicAdd(S.S + (size_t)i * G.nv + v, dn);
}

// BP of the residual change of the pair's rows into g_J, and r~^J = r.
template <typename T>
__device__ __forceinline__ void bp_solve_body(const DeviceGeom &G, const SolveDev &S, int tile,
                                              int slot, int p) {
    int a, i, j, u, v;
    bool act;
    if (!solve_pixel(G, S, tile, slot, p, a, i, j, u, v, act) || !act) return;
    if (S.owned && !S.owned[j]) return;   // another process owns block j
    const int64_t row = ((int64_t)a * G.nv + v) * G.nu + u;
    const T *r = reinterpret_cast<const T *>(S.r);
    T *rt = reinterpret_cast<T *>(S.rt);
    bool in;
    const int64_t kt = zslot(G, j, a, u, v, in);
    const float rv = ldv(r + row), ro = ldv(rt + kt);
    stf(rt + kt, rv);
    const float dw = rv - ro;
    if (dw == 0.f) return;
    const bool yf = S.gT != nullptr && G.view_yfast[a];
    float *dst = yf ? S.gT : S.g;
    RayWalk w;
    if (!ray_setup(G, a, u, v, G.plane_start[j], G.plane_start[j + 1], w, yf)) return;
    const float wl = dw * w.L;
    ray_walk_fast(w, [&](int idx, float s) {
        if (s > 0.f) atomicAdd(dst + idx, s * wl);
    });
}

// FP, residual and BP of one ray in one pass (one column block per iteration):
// the ray's BP weight r_new - r~ depends only on its own FP, so the back
// projection follows the forward walk without waiting for other rays.
template <typename T>
__device__ __forceinline__ void fpbp_solve_body(const DeviceGeom &G, const SolveDev &S,
                                                const T *__restrict__ x, int tile, int slot, int p) {
    int a, i, j, u, v;
    bool act;
    if (!solve_pixel(G, S, tile, slot, p, a, i, j, u, v, act)) return;
    const int plo = G.plane_start[j], phi = G.plane_start[j + 1];
    const bool yf = act && S.xT != nullptr && G.view_yfast[a];
    float zn = 0.f;
    if (act) {
        const T *src = yf ? reinterpret_cast<const T *>(S.xT) : x;
        RayWalk w;
        if (ray_setup(G, a, u, v, plo, phi, w, yf)) {
            float acc = 0.f;
            ray_walk_fast(w, [&](int idx, float s) { acc = fmaf(s, ldf(src + idx), acc); });
            zn = acc * w.L;
        }
    }
    const int64_t row = act ? ((int64_t)a * G.nv + v) * G.nu + u : 0;
    T *z = reinterpret_cast<T *>(S.z);
    double dn = 0.0;
    float dw = 0.f;
    if (act) {
        bool in;
        const int64_t kj = zslot(G, j, a, u, v, in);
        stf(z + kj, zn);
        zn = rnd(zn, z);
        float zs = 0.f;
        for (int jj = 0; jj < G.N; ++jj) {   // z^jj is 0 outside block jj's band
            if (jj == j) {
                zs += zn;
                continue;
            }
            const int64_t k = zslot(G, jj, a, u, v, in);
            if (in) zs += ldv(z + k);
        }
        T *r = reinterpret_cast<T *>(S.r);
        T *rt = reinterpret_cast<T *>(S.rt);
        const float rn = rnd(ldf(reinterpret_cast<const T *>(S.y) + row) - zs, r);
        const float ro = ldv(r + row);
        stf(r + row, rn);
        dn = (double)rn * rn - (double)ro * ro;
        dw = rn - ldv(rt + kj);
        stf(rt + kj, rn);
    }
    for (int o = 16; o > 0; o >>= 1) dn += __shfl_xor_sync(0xffffffffu, dn, o);
    if ((threadIdx.x & 31) == 0 && act && dn != 0.0) atomicAdd(S.S + (size_t)i * G.nv + v, dn);
    if (!act || dw == 0.f) return;
    float *dst = (S.gT != nullptr && G.view_yfast[a]) ? S.gT : S.g;
    RayWalk w;
    if (!ray_setup(G, a, u, v, plo, phi, w, S.gT != nullptr && G.view_yfast[a])) return;
    const float wl = dw * w.L;
    ray_walk_fast(w, [&](int idx, float s) {
        if (s > 0.f) atomicAdd(dst + idx, s * wl);
    });
}

template <typename T>
__global__ void __launch_bounds__(128) fpbp_solve_kernel(const DeviceGeom G, const SolveDev S,
                                                         const T *__restrict__ x) {
    fpbp_solve_body<T>(G, S, x, blockIdx.x / G.max_views, blockIdx.x % G.max_views, blockIdx.z);
}

// FP, residual and BP of one ray in one pass when an iteration selects several
// column blocks (at most NC) for each selected row block: the ray's new
// residual needs the new z^j of every selected block, so the thread walks each
// selected slab forward, forms r = y - sum_j z^j, then walks each slab back
// with that block's own snapshot difference r - r~^j. With detector cells
// (Algorithm 2) a block's walks are taken only by the rays of the cell drawn
// for that pair; the others keep their z^j and r~^j. The work item is a tile
// of the bounding box of the selected blocks' bands (the rows the split path's
// residual pass covers) for one view of one selected row block (rs).
template <typename T, int NC>
__device__ __forceinline__ void fpbpm_solve_body(const DeviceGeom &G, const SolveDev &S,
                                                 const T *__restrict__ x, int tile, int slot,
                                                 int rs) {
    const Work &W = *S.work;
    if (rs >= W.n_rows) return;
    const int i = W.rows[rs];
    if (slot >= G.block_nviews[i]) return;
    const int a = G.block_views[i * G.max_views + slot];
    int js[NC];
    Band b{1 << 30, -1, 1 << 30, -1};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        js[c] = c < W.n_cols ? W.cols[c] : -1;
        if (js[c] < 0) continue;
        const Band q = G.bands[(size_t)a * (G.N + 1) + js[c]];
        if (q.u0 > q.u1 || q.v0 > q.v1) continue;
        b.u0 = min(b.u0, q.u0);
        b.u1 = max(b.u1, q.u1);
        b.v0 = min(b.v0, q.v0);
        b.v1 = max(b.v1, q.v1);
    }
    int u, v, nt;
    const bool act = G.nv > 1 ? tile_pixel<true>(b, tile, u, v, nt) : tile_pixel<false>(b, tile, u, v, nt);
    if (tile >= nt) return;   // uniform over the CTA
    const bool yf = S.xT != nullptr && G.view_yfast[a];
    const T *src = yf ? reinterpret_cast<const T *>(S.xT) : x;
    T *z = reinterpret_cast<T *>(S.z);
    float zn[NC];
    int64_t kj[NC];
    bool inb[NC], part[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        zn[c] = 0.f;
        inb[c] = part[c] = false;
        kj[c] = 0;
        if (!act || js[c] < 0) continue;
        kj[c] = zslot(G, js[c], a, u, v, inb[c]);
        // the ray takes part in pair (i, j) if it lies in j's band (z^j is 0
        // outside it) and in the detector cell drawn for the pair at this view
        // (pairs are the drawn rows x the drawn columns, row-major)
        part[c] = inb[c];
        if (part[c] && S.n_cells > 1) {
            const int cell = S.cells[(rs * W.n_cols + c) * G.max_views + slot];
            if (cell >= 0)
                part[c] = ((cell & 1) != 0) == (u >= G.nu / 2) &&
                          (S.n_cells != 4 || ((cell >> 1) != 0) == (v >= G.nv / 2));
        }
        if (!part[c]) continue;
        RayWalk w;
        if (ray_setup(G, a, u, v, G.plane_start[js[c]], G.plane_start[js[c] + 1], w, yf)) {
            float acc = 0.f;
            ray_walk_fast(w, [&](int idx, float s) { acc = fmaf(s, ldf(src + idx), acc); });
            zn[c] = acc * w.L;
        }
        stf(z + kj[c], zn[c]);
        zn[c] = rnd(zn[c], z);
    }
    // a ray that takes part in no pair kept every z^j, so its r stands
    bool any = false;
#pragma unroll
    for (int c = 0; c < NC; ++c) any |= part[c];
    const int64_t row = act ? ((int64_t)a * G.nv + v) * G.nu + u : 0;
    T *r = reinterpret_cast<T *>(S.r);
    double dn = 0.0;
    float rn = 0.f;
    if (act && any) {
        float zs = 0.f;
        for (int jj = 0; jj < G.N; ++jj) {   // z^jj is 0 outside block jj's band
            bool sel = false;
            float zv = 0.f;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (jj == js[c] && part[c]) {
                    sel = true;
                    zv = zn[c];
                }
            if (sel) {
                zs += zv;
                continue;
            }
            bool inj;
            const int64_t k = zslot(G, jj, a, u, v, inj);
            if (inj) zs += ldv(z + k);
        }
        rn = rnd(ldf(reinterpret_cast<const T *>(S.y) + row) - zs, r);
        const float ro = ldv(r + row);
        stf(r + row, rn);
        dn = (double)rn * rn - (double)ro * ro;
    }
    // the 32 lanes of a warp share one detector row; lane 0 has the lowest u,
    // so it is active whenever any lane of the warp is
    for (int o = 16; o > 0; o >>= 1) dn += __shfl_xor_sync(0xffffffffu, dn, o);
    if ((threadIdx.x & 31) == 0 && act && dn != 0.0) atomicAdd(S.S + (size_t)i * G.nv + v, dn);
    const bool yb = S.gT != nullptr && G.view_yfast[a];
    float *dst = yb ? S.gT : S.g;
    T *rt = reinterpret_cast<T *>(S.rt);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (!act || !part[c]) continue;
        const float dw = rn - ldv(rt + kj[c]);
        stf(rt + kj[c], rn);
        if (dw == 0.f) continue;
        RayWalk w;
        if (!ray_setup(G, a, u, v, G.plane_start[js[c]], G.plane_start[js[c] + 1], w, yb)) continue;
        const float wl = dw * w.L;
        ray_walk_fast(w, [&](int idx, float s) {
            if (s > 0.f) atomicAdd(dst + idx, s * wl);
        });
    }
}

template <typename T, int NC>
__global__ void __launch_bounds__(128) fpbpm_solve_kernel(const DeviceGeom G, const SolveDev S,
                                                          const T *__restrict__ x) {
    fpbpm_solve_body<T, NC>(G, S, x, blockIdx.x / G.max_views, blockIdx.x % G.max_views, blockIdx.z);
}

template <typename T, bool FUSED>
__global__ void __launch_bounds__(128) fp_solve_kernel(const DeviceGeom G, const SolveDev S,
                                                       const T *__restrict__ x) {
    fp_solve_body<T, FUSED>(G, S, x, blockIdx.x / G.max_views, blockIdx.x % G.max_views, blockIdx.z);
}

template <typename T>
__global__ void __launch_bounds__(128) bp_solve_kernel(const DeviceGeom G, const SolveDev S) {
    bp_solve_body<T>(G, S, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// Warm start (a starting image x0 != 0): z^j = A^j x0_J for every row of every
// block's band, then r = y - sum_j z^j. Every kernel returns at once when the
// flag says x0 is zero, so Algorithm 1's own start costs one read of the image.

template <typename T>
__global__ void __launch_bounds__(256) nonzero_kernel(const T *__restrict__ x, int64_t n,
                                                      int *__restrict__ flag) {
    bool nz = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        nz |= ldf(x + k) != 0.f;
    if (__syncthreads_or(nz) && threadIdx.x == 0) *flag = 1;
}

// z^j of every block at every view: work items (block, view, tile of the
// view's band) taken in turn by a grid of a few CTAs per SM.
template <bool k3D, typename T>
__global__ void __launch_bounds__(128) warm_fp_kernel(const DeviceGeom G, int tiles,
                                                      const T *__restrict__ x,
                                                      const T *__restrict__ xT, T *__restrict__ z,
                                                      const int *__restrict__ flag) {
    if (*flag == 0) return;
    const int64_t total = (int64_t)G.N * G.n_views * tiles;
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int tile = (int)(item % tiles);
        const int64_t ja = item / tiles;
        const int a = (int)(ja % G.n_views), j = (int)(ja / G.n_views);
        const Band b = G.bands[(size_t)a * (G.N + 1) + j];
        int u, v, nt;
        if (!tile_pixel<k3D>(b, tile, u, v, nt)) continue;
        const bool yf = xT != nullptr && G.view_yfast[a];
        const T *src = yf ? xT : x;
        RayWalk w;
        float acc = 0.f;
        if (ray_setup(G, a, u, v, G.plane_start[j], G.plane_start[j + 1], w, yf)) {
            ray_walk_fast(w, [&](int idx, float s) { acc = fmaf(s, ldf(src + idx), acc); });
            acc *= w.L;
        }
        bool in;
        stf(z + zslot(G, j, a, u, v, in), acc);
    }
}

// r = y - sum_j z^j over every row, the blocks summed in block order as in the
// solver's FP epilogue (z^j is 0 outside block j's band).
template <typename T>
__global__ void __launch_bounds__(256) warm_residual_kernel(const DeviceGeom G,
                                                            const T *__restrict__ y,
                                                            const T *__restrict__ z,
                                                            T *__restrict__ r,
                                                            const int *__restrict__ flag) {
    if (*flag == 0) return;
    const int64_t n = (int64_t)G.n_views * G.nv * G.nu;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(row % G.nu);
        const int64_t av = row / G.nu;
        const int v = (int)(av % G.nv), a = (int)(av / G.nv);
        float zs = 0.f;
        for (int jj = 0; jj < G.N; ++jj) {
            bool in;
            const int64_t k = zslot(G, jj, a, u, v, in);
            if (in) zs += ldf(z + k);
        }
        stf(r + row, ldf(y + row) - zs);
    }
}

// ---------------------------------------------------------------------------
// Serving rounds: persistent kernels over the work items of every resident
// request (one CTA work item = one detector tile of one view of one pair).
// Items are handed out by an atomic counter, so requests of very different
// sizes share the GPU without a per-request launch.

__device__ __forceinline__ int round_entry(const ReqDesc *T, int lo, int hi, long long item) {
    int r = lo;
    while (r + 1 < hi && T[r + 1].work_begin <= item) ++r;
    return r;
}

// The request table of one server per device in constant memory: the
// persistent passes read a request's geometry and solver arguments through
// the constant cache, as the plain kernels read their parameters (a lone
// 256^3 request served: 76 against 99 ms for two epochs with the arguments
// staged in shared memory). Other servers on the same device use the table in
// global memory.
__constant__ ReqDesc c_round_table[kRoundConstSlots];

bsgd_status upload_round_const_table(const ReqDesc *h, int n, cudaStream_t st) {
    if (n > kRoundConstSlots) return fail(BSGD_ERR_INVALID_ARG, "too many entries for the constant table");
    if (n > 0)
        BSGD_CUDA(cudaMemcpyToSymbolAsync(c_round_table, h, sizeof(ReqDesc) * n, 0,
                                          cudaMemcpyHostToDevice, st));
    return BSGD_OK;
}

// Persistent kernel of one class of requests (MULTI: several column blocks
// per iteration; T: storage type): CTA-sized work items (one detector tile of
// one view of one pair, or of one drawn row block with several column blocks)
// handed out by the class's atomic counter. CT: the table is c_round_table;
// otherwise it is T_ in global memory, and a CTA copies the request's
// geometry and solver arguments into shared memory when it moves to another
// request, so that they do not compete with the gathers for L1.
template <bool MULTI, typename T, bool CT>
__global__ void __launch_bounds__(128, CT ? 1 : (MULTI ? 7 : 10))
    round_solve_kernel(const ReqDesc *__restrict__ T_, RoundCtl *__restrict__ C) {
    constexpr int CLS = 3 * (MULTI ? 1 : 0) + (sizeof(T) == 4 ? BSGD_F32
                                               : std::is_same<T, __nv_bfloat16>::value ? BSGD_BF16
                                                                                       : BSGD_F16);
    __shared__ long long s_item;
    __shared__ DeviceGeom sG;
    __shared__ SolveDev sS;
    static_assert(sizeof(DeviceGeom) % 4 == 0 && sizeof(SolveDev) % 4 == 0, "word copies");
    const int lo = C->lo[CLS], hi = C->hi[CLS];
    const unsigned long long round = C->round;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(&C->next[CLS], 1ull);
        __syncthreads();   // the previous item is done with sG / sS; s_item is visible
        const long long item = s_item;
        if (item >= C->total_items[CLS] || lo >= hi) return;
        if (CT) {
            int e = lo;
            while (e + 1 < hi && c_round_table[e + 1].work_begin <= item) ++e;
            const ReqDesc &q = c_round_table[e];
            __syncthreads();   // every thread has read s_item
            if (!q.active || round_skips(q.period, round) || item >= q.work_begin + q.work_count) continue;
            long long local = item - q.work_begin;
            const int slot = (int)(local % q.G.max_views);
            local /= q.G.max_views;
            const int tile = (int)(local % q.max_tiles);
            const int p = (int)(local / q.max_tiles);
            const T *x = reinterpret_cast<const T *>(q.x);
            if (!MULTI) fpbp_solve_body<T>(q.G, q.S, x, tile, slot, p);
            else if (q.kN <= 2) fpbpm_solve_body<T, 2>(q.G, q.S, x, tile, slot, p);
            else fpbpm_solve_body<T, 4>(q.G, q.S, x, tile, slot, p);
            continue;
        }
        const int e = round_entry(T_, lo, hi, item);
        const ReqDesc &q = T_[e];
        if (e != cur) {
            const uint32_t *gsrc = reinterpret_cast<const uint32_t *>(&q.G);
            const uint32_t *ssrc = reinterpret_cast<const uint32_t *>(&q.S);
            uint32_t *gdst = reinterpret_cast<uint32_t *>(&sG), *sdst = reinterpret_cast<uint32_t *>(&sS);
            for (int k = threadIdx.x; k < (int)(sizeof(DeviceGeom) / 4); k += blockDim.x) gdst[k] = gsrc[k];
            for (int k = threadIdx.x; k < (int)(sizeof(SolveDev) / 4); k += blockDim.x) sdst[k] = ssrc[k];
            cur = e;
        }
        const int active = q.active && !round_skips(q.period, round), max_tiles = q.max_tiles, kN = q.kN;
        const int64_t wb = q.work_begin, wc = q.work_count;
        const T *x = reinterpret_cast<const T *>(q.x);
        __syncthreads();   // sG / sS are complete; every thread has read s_item
        if (!active || item >= wb + wc) continue;
        long long local = item - wb;
        const int slot = (int)(local % sG.max_views);
        local /= sG.max_views;
        const int tile = (int)(local % max_tiles);
        const int p = (int)(local / max_tiles);   // pair (one block) or row-block slot
        if (!MULTI) fpbp_solve_body<T>(sG, sS, x, tile, slot, p);
        else if (kN <= 2) fpbpm_solve_body<T, 2>(sG, sS, x, tile, slot, p);
        else fpbpm_solve_body<T, 4>(sG, sS, x, tile, slot, p);
    }
}

namespace {
template <bool MULTI, typename T, bool CT>
const void *round_kernel_ptr() { return (const void *)round_solve_kernel<MULTI, T, CT>; }
template <bool CT>
const void *round_kernel_of(int cls) {
    switch (cls) {
    case 0: return round_kernel_ptr<false, float, CT>();
    case 1: return round_kernel_ptr<false, __nv_bfloat16, CT>();
    case 2: return round_kernel_ptr<false, __half, CT>();
    case 3: return round_kernel_ptr<true, float, CT>();
    case 4: return round_kernel_ptr<true, __nv_bfloat16, CT>();
    default: return round_kernel_ptr<true, __half, CT>();
    }
}
const void *round_kernel(int cls, bool ct) { return ct ? round_kernel_of<true>(cls) : round_kernel_of<false>(cls); }
}  // namespace

int round_persistent_grid(int cls, bool ct) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, round_kernel(cls, ct), 128, 0);
    cudaGetLastError();
    return sms * std::max(1, a);
}

bsgd_status launch_round_solve(const ReqDesc *table, RoundCtl *ctl, int cls, bool ct, int grid,
                               cudaStream_t st) {
    void *args[] = {(void *)&table, (void *)&ctl};
    BSGD_CUDA(cudaLaunchKernel(round_kernel(cls, ct), dim3(grid), dim3(128), args, 0, st));
    return BSGD_OK;
}

// ---------------------------------------------------------------------------
// Host launchers

namespace {

RowSel all_rows(const bsgd_geometry *g) {
    RowSel R{};
    R.n = g->M;
    for (int i = 0; i < g->M && i < 64; ++i) R.ids[i] = i;
    return R;
}

template <typename F>
bsgd_status for_row_chunks(const bsgd_geometry *g, const PlainLaunch &L, F &&f) {
    // row-block ids in chunks of 64 per launch
    (void)g;
    RowSel R{};
    int k = 0;
    for (int t = 0; t < L.n_rb; ++t) {
        R.ids[k++] = L.row_ids[t];
        if (k == 64 || t == L.n_rb - 1) {
            R.n = k;
            BSGD_TRY(f(R));
            k = 0;
        }
    }
    return BSGD_OK;
}

std::vector<int> views_of(const bsgd_geometry *g, const RowSel &R) {
    std::vector<int> v;
    for (int k = 0; k < R.n; ++k)
        for (int a : g->block_views[R.ids[k]]) v.push_back(a);
    return v;
}

template <typename TX, typename TY>
void fp_plain_go(const bsgd_geometry *g, dim3 grid, const RowSel &R, int j0, int j1, const void *x,
                 void *y, const void *xT, cudaStream_t st) {
    if (g->desc.nv > 1)
        fp_plain_kernel<true, TX, TY><<<grid, 128, 0, st>>>(g->dg, R, j0, j1, (const TX *)x, (TY *)y,
                                                            (const TX *)xT);
    else
        fp_plain_kernel<false, TX, TY><<<grid, 128, 0, st>>>(g->dg, R, j0, j1, (const TX *)x, (TY *)y,
                                                             (const TX *)xT);
}

template <typename TX>
void fp_plain_y(const bsgd_geometry *g, dim3 grid, const RowSel &R, int j0, int j1, const void *x,
                void *y, bsgd_dtype yt, const void *xT, cudaStream_t st) {
    if (yt == BSGD_F32) fp_plain_go<TX, float>(g, grid, R, j0, j1, x, y, xT, st);
    else if (yt == BSGD_BF16) fp_plain_go<TX, __nv_bfloat16>(g, grid, R, j0, j1, x, y, xT, st);
    else fp_plain_go<TX, __half>(g, grid, R, j0, j1, x, y, xT, st);
}

// Grid of the plane-tile kernels: 32 x 32 tiles over the planes, at most 16
// CTAs of 256 threads per SM.
int plane_tile_grid(const bsgd_geometry *g, int z0, int z1) {
    const int64_t t = (int64_t)((g->desc.nx + 31) / 32) * ((g->desc.ny + 31) / 32) * (z1 - z0);
    return (int)std::max<int64_t>(1, std::min<int64_t>(t, 152 * 8));
}

}  // namespace

bsgd_status zero_rows(const bsgd_geometry *g, const int *row_ids, int n_rb, void *y,
                      bsgd_dtype yt, cudaStream_t st) {
    PlainLaunch L{row_ids, n_rb, 0, g->N, 0};
    return for_row_chunks(g, L, [&](const RowSel &R) -> bsgd_status {
        dim3 grid(std::max(1, (int)std::min<int64_t>(64, ((int64_t)g->desc.nu * g->desc.nv * 2 + 511) / 512)),
                  R.n * g->max_views);
        zero_views_kernel<<<grid, 128, 0, st>>>(g->dg, R, y, (int)dtype_size(yt));
        BSGD_CUDA(cudaGetLastError());
        return BSGD_OK;
    });
}

bool plain_wants_transpose(const bsgd_geometry *g, const int *row_ids, int n_rb) {
    if (g->desc.nz <= 1) return false;
    for (int k = 0; k < n_rb; ++k)
        for (int a : g->block_views[row_ids[k]])
            if (g->view_yfast[a]) return true;
    return false;
}

bsgd_status plain_transpose(const bsgd_geometry *g, const void *x, bsgd_dtype xt, void *xT, int j0,
                            int j1, cudaStream_t st) {
    const int z0 = g->plane_start[j0], z1 = g->plane_start[j1];
    if (z1 <= z0) return BSGD_OK;
    const int gb = plane_tile_grid(g, z0, z1);
    if (xt == BSGD_F32)
        transpose_planes_kernel<float><<<gb, 256, 0, st>>>(g->dg, z0, z1, (const float *)x, (float *)xT);
    else if (xt == BSGD_BF16)
        transpose_planes_kernel<__nv_bfloat16><<<gb, 256, 0, st>>>(
            g->dg, z0, z1, (const __nv_bfloat16 *)x, (__nv_bfloat16 *)xT);
    else
        transpose_planes_kernel<__half><<<gb, 256, 0, st>>>(g->dg, z0, z1, (const __half *)x, (__half *)xT);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status plain_add_transposed(const bsgd_geometry *g, const float *gT, float *x, int j0, int j1,
                                 cudaStream_t st) {
    const int z0 = g->plane_start[j0], z1 = g->plane_start[j1];
    if (z1 <= z0) return BSGD_OK;
    add_transposed_kernel<<<plane_tile_grid(g, z0, z1), 256, 0, st>>>(g->dg, z0, z1, gT, x);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status launch_fp_plain(const bsgd_geometry *g, const PlainLaunch &L, const void *x,
                            bsgd_dtype xt, void *y, bsgd_dtype yt, int accumulate,
                            cudaStream_t st, const void *xT) {
    (void)accumulate;
    return for_row_chunks(g, L, [&](const RowSel &R) -> bsgd_status {
        const int tiles = tiles_for(g, views_of(g, R), L.j0, L.j1, tile_u(g), tile_v(g));
        if (tiles == 0) return BSGD_OK;
        const int64_t ctas = (int64_t)tiles * R.n * g->max_views;
        if (ctas > 0x7fffffff) return fail(BSGD_ERR_INVALID_ARG, "forward projection grid too large");
        dim3 grid((unsigned)ctas);
        if (xt == BSGD_F32) fp_plain_y<float>(g, grid, R, L.j0, L.j1, x, y, yt, xT, st);
        else if (xt == BSGD_BF16) fp_plain_y<__nv_bfloat16>(g, grid, R, L.j0, L.j1, x, y, yt, xT, st);
        else fp_plain_y<__half>(g, grid, R, L.j0, L.j1, x, y, yt, xT, st);
        BSGD_CUDA(cudaGetLastError());
        return BSGD_OK;
    });
}

bsgd_status launch_bp_plain(const bsgd_geometry *g, const PlainLaunch &L, const void *r,
                            bsgd_dtype rt, float *x, float scale, cudaStream_t st, float *gT) {
    return for_row_chunks(g, L, [&](const RowSel &R) -> bsgd_status {
        const int tiles = tiles_for(g, views_of(g, R), L.j0, L.j1, tile_u(g), tile_v(g));
        if (tiles == 0) return BSGD_OK;
        dim3 grid(tiles, R.n * g->max_views);
        const bool t3 = g->desc.nv > 1;
#define BP_GO(T)                                                                                   \
    if (t3) bp_plain_kernel<true, T><<<grid, 128, 0, st>>>(g->dg, R, L.j0, L.j1, (const T *)r, x, scale, gT); \
    else bp_plain_kernel<false, T><<<grid, 128, 0, st>>>(g->dg, R, L.j0, L.j1, (const T *)r, x, scale, gT);
        if (rt == BSGD_F32) { BP_GO(float) }
        else if (rt == BSGD_BF16) { BP_GO(__nv_bfloat16) }
        else { BP_GO(__half) }
#undef BP_GO
        BSGD_CUDA(cudaGetLastError());
        return BSGD_OK;
    });
}

bsgd_status launch_count(const bsgd_geometry *g, const PlainLaunch &L,
                         unsigned long long *d_counts, cudaStream_t st) {
    return for_row_chunks(g, L, [&](const RowSel &R) -> bsgd_status {
        const int tiles = tiles_for(g, views_of(g, R), L.j0, L.j1, tile_u(g), tile_v(g));
        if (tiles == 0) return BSGD_OK;
        dim3 grid(tiles, R.n * g->max_views);
        if (g->desc.nv > 1) count_kernel<true><<<grid, 128, 0, st>>>(g->dg, R, L.j0, L.j1, 1, d_counts);
        else count_kernel<false><<<grid, 128, 0, st>>>(g->dg, R, L.j0, L.j1, 1, d_counts);
        BSGD_CUDA(cudaGetLastError());
        return BSGD_OK;
    });
}

bsgd_status launch_count_cells(const bsgd_geometry *g, int j, int n_cells,
                               unsigned long long *d_counts, cudaStream_t st) {
    const RowSel R = all_rows(g);
    std::vector<int> all(g->desc.n_views);
    for (int a = 0; a < g->desc.n_views; ++a) all[a] = a;
    const int tiles = tiles_for(g, all, j, j + 1, tile_u(g), tile_v(g));
    if (tiles == 0) return BSGD_OK;
    if (g->M > 64) return fail(BSGD_ERR_INVALID_ARG, "M > 64 not supported by the counter");
    dim3 grid(tiles, R.n * g->max_views);
    if (g->desc.nv > 1) count_kernel<true><<<grid, 128, 0, st>>>(g->dg, R, j, j + 1, n_cells, d_counts);
    else count_kernel<false><<<grid, 128, 0, st>>>(g->dg, R, j, j + 1, n_cells, d_counts);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status launch_fp_solve(const bsgd_geometry *g, const SolveDev &S, const void *x,
                            bsgd_dtype st_t, int max_pairs, int max_tiles, bool fused,
                            cudaStream_t st) {
    // view slot fastest: CTAs running together hold the same band rows of
    // every view, and a launch ends on the band's last (edge) rows
    dim3 grid((unsigned)max_tiles * g->max_views, 1, max_pairs);
#define FPS_GO(T)                                                                          \
    if (fused) fp_solve_kernel<T, true><<<grid, 128, 0, st>>>(g->dg, S, (const T *)x);     \
    else fp_solve_kernel<T, false><<<grid, 128, 0, st>>>(g->dg, S, (const T *)x);
    if (st_t == BSGD_F32) { FPS_GO(float) }
    else if (st_t == BSGD_BF16) { FPS_GO(__nv_bfloat16) }
    else { FPS_GO(__half) }
#undef FPS_GO
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status launch_fpbp_solve(const bsgd_geometry *g, const SolveDev &S, const void *x,
                              bsgd_dtype st_t, int max_pairs, int max_tiles, cudaStream_t st) {
    // view slot fastest: CTAs running together hold the same band rows of
    // every view, and a launch ends on the band's last (edge) rows
    dim3 grid((unsigned)max_tiles * g->max_views, 1, max_pairs);
    if (st_t == BSGD_F32) fpbp_solve_kernel<float><<<grid, 128, 0, st>>>(g->dg, S, (const float *)x);
    else if (st_t == BSGD_BF16) fpbp_solve_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(g->dg, S, (const __nv_bfloat16 *)x);
    else fpbp_solve_kernel<__half><<<grid, 128, 0, st>>>(g->dg, S, (const __half *)x);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status launch_fpbpm_solve(const bsgd_geometry *g, const SolveDev &S, const void *x,
                               bsgd_dtype st_t, int max_rows, int max_tiles, int n_cols,
                               cudaStream_t st) {
    if (n_cols < 2 || n_cols > kMaxFusedCols)
        return fail(BSGD_ERR_INVALID_ARG, "fused multi-block pass takes 2 to 4 column blocks");
    // view slot fastest, as in the one-block fused kernel
    dim3 grid((unsigned)max_tiles * g->max_views, 1, max_rows);
#define FPBPM_GO(T, NC) fpbpm_solve_kernel<T, NC><<<grid, 128, 0, st>>>(g->dg, S, (const T *)x);
#define FPBPM_T(T) if (n_cols <= 2) { FPBPM_GO(T, 2) } else { FPBPM_GO(T, 4) }
    if (st_t == BSGD_F32) { FPBPM_T(float) }
    else if (st_t == BSGD_BF16) { FPBPM_T(__nv_bfloat16) }
    else { FPBPM_T(__half) }
#undef FPBPM_T
#undef FPBPM_GO
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status launch_nonzero(const bsgd_geometry *g, const void *x, bsgd_dtype st_t, int *flag,
                           cudaStream_t st) {
    const int64_t C = g->n_cols();
    BSGD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    const int gn = (int)std::max<int64_t>(1, std::min<int64_t>((C + 255) / 256, 152 * 8));
    if (st_t == BSGD_F32) nonzero_kernel<float><<<gn, 256, 0, st>>>((const float *)x, C, flag);
    else if (st_t == BSGD_BF16) nonzero_kernel<__nv_bfloat16><<<gn, 256, 0, st>>>((const __nv_bfloat16 *)x, C, flag);
    else nonzero_kernel<__half><<<gn, 256, 0, st>>>((const __half *)x, C, flag);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status launch_warm_start(const bsgd_geometry *g, const SolveDev &S, const void *x,
                              bsgd_dtype st_t, int *flag, cudaStream_t st) {
    const int64_t C = g->n_cols(), R = g->n_rows();
    BSGD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    const int gn = (int)std::max<int64_t>(1, std::min<int64_t>((C + 255) / 256, 152 * 8));
    const int gr = (int)std::max<int64_t>(1, std::min<int64_t>((R + 255) / 256, 152 * 8));
    std::vector<int> all(g->desc.n_views);
    for (int a = 0; a < g->desc.n_views; ++a) all[a] = a;
    int tiles = 0;   // the most tiles any (view, block) band needs
    for (int j = 0; j < g->N; ++j) tiles = std::max(tiles, tiles_for(g, all, j, j + 1, tile_u(g), tile_v(g)));
    const int gw = 152 * 8;
    const bool t3 = g->desc.nv > 1;
#define WARM_GO(T)                                                                                 \
    {                                                                                              \
        nonzero_kernel<T><<<gn, 256, 0, st>>>((const T *)x, C, flag);                             \
        if (tiles > 0) {                                                                           \
            if (t3) warm_fp_kernel<true, T><<<gw, 128, 0, st>>>(g->dg, tiles, (const T *)x,        \
                                                                (const T *)S.xT, (T *)S.z, flag);  \
            else warm_fp_kernel<false, T><<<gw, 128, 0, st>>>(g->dg, tiles, (const T *)x,          \
                                                              (const T *)S.xT, (T *)S.z, flag);    \
        }                                                                                          \
        warm_residual_kernel<T><<<gr, 256, 0, st>>>(g->dg, (const T *)S.y, (const T *)S.z,         \
                                                    (T *)S.r, flag);                               \
    }
    if (st_t == BSGD_F32) WARM_GO(float)
    else if (st_t == BSGD_BF16) WARM_GO(__nv_bfloat16)
    else WARM_GO(__half)
#undef WARM_GO
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status launch_bp_solve(const bsgd_geometry *g, const SolveDev &S, bsgd_dtype st_t,
                            int max_pairs, int max_tiles, cudaStream_t st) {
    // tile fastest: the BP alone scatters faster when the CTAs running
    // together hold different views (their atomics spread over more of g);
    // the FP and the fused kernel gather faster with the view slot fastest
    dim3 grid(max_tiles, g->max_views, max_pairs);
    if (st_t == BSGD_F32) bp_solve_kernel<float><<<grid, 128, 0, st>>>(g->dg, S);
    else if (st_t == BSGD_BF16) bp_solve_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(g->dg, S);
    else bp_solve_kernel<__half><<<grid, 128, 0, st>>>(g->dg, S);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

}  // namespace bsgd
