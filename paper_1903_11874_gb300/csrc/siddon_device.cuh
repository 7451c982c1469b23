// Device-side Siddon traversal shared by the projector kernels.
//
// A_ij is the length of ray i inside voxel j (Sec. 1, after Eq. 1), computed on
// the fly. The walk is the incremental form of Siddon's method (Jacobs et al.,
// the variant the paper cites): after clipping the ray to the box of the column
// block, it keeps the parameter of the next x, y and z plane crossing and steps
// into the neighbouring voxel across whichever plane comes first.
//
// Precision choices (FP32 throughout):
//   * detector pixels are addressed by their offset from the detector centre,
//     which FP32 holds exactly, so a central row or column that lies in a voxel
//     face stays exactly in it;
//   * the walk carries, per axis, the parameter left to the next plane: numbers
//     of the size of one voxel's crossing, reset exactly at every crossing, so
//     the rounding of a boundary is a small fraction of a voxel instead of an
//     ulp of the whole ray length;
//   * per-axis crossing counts come from the entry and exit voxels, so the walk
//     never leaves the box whatever the rounding, and no segment is negative.
#pragma once

#include "bsgd_internal.h"

namespace bsgd {

__device__ __forceinline__ float ldf(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ldf(const __half *p) { return __half2float(__ldg(p)); }
// coherent loads for data that an earlier kernel of the same step wrote
__device__ __forceinline__ float ldv(const float *p) { return *p; }
__device__ __forceinline__ float ldv(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ldv(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void stf(float *p, float v) { *p = v; }
__device__ __forceinline__ void stf(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void stf(__half *p, float v) { *p = __float2half_rn(v); }
// the value a store of v reads back as (storage rounding)
__device__ __forceinline__ float rnd(float v, const float *) { return v; }
__device__ __forceinline__ float rnd(float v, const __nv_bfloat16 *) {
    return __bfloat162float(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float rnd(float v, const __half *) {
    return __half2float(__float2half_rn(v));
}

constexpr float kInf = __builtin_huge_valf();

// Index of row (a, u, v) in block j's compact sinogram (z^j, r~^j); `in`
// tells whether the row lies in the block's band (outside it the value is 0).
__device__ __forceinline__ int64_t zslot(const DeviceGeom &G, int j, int a, int u, int v, bool &in) {
    const Band b = G.bands[(size_t)a * (G.N + 1) + j];
    in = u >= b.u0 && u <= b.u1 && v >= b.v0 && v <= b.v1;
    return G.zoff[(size_t)j * G.n_views + a] + (int64_t)(v - b.v0) * (b.u1 - b.u0 + 1) + (u - b.u0);
}

struct RayWalk {
    float tx, ty, tz;   // parameter left to the next interior plane per axis (INF: none)
    float te;           // parameter left to the exit face (INF until the exit axis has
                        // crossed its last interior plane)
    float Dx, Dy, Dz;   // parameter between two planes of each axis (|1 / d|)
    int cx, cy, cz;     // interior planes left to cross per axis
    int ex;             // axis whose face the ray leaves the box through
    int sx, sy, sz;     // flat voxel index step per axis
    int idx;            // current voxel (flat index in the whole volume)
    int n;              // interior crossings = voxels to visit - 1
    float L;            // |d| in mm: segment length = parameter difference * L
    float fin;          // parameter from the last interior crossing to the exit face
    unsigned vmax;      // largest flat voxel index of the volume
};

// Clip one axis: narrows [amin, amax] and records which axis sets the exit;
// false if the ray is parallel to the axis and outside the slab (a ray lying in
// a face belongs to the + side).
__device__ __forceinline__ bool clip_axis(float q0, float d, float lo, float hi, int axis,
                                          float &amin, float &amax, int &exit_axis) {
    if (d != 0.f) {
        const float inv = 1.0f / d;
        const float t0 = (lo - q0) * inv, t1 = (hi - q0) * inv;
        amin = fmaxf(amin, fminf(t0, t1));
        const float te = fmaxf(t0, t1);
        if (te < amax) {
            amax = te;
            exit_axis = axis;
        }
        return true;
    }
    return q0 >= lo && q0 < hi;
}

// Entry / exit voxel along one axis and the parameter to its first plane.
// The entry fraction is fma(amin, d, q0 - i): q0 - i is exact (an integer off a
// float of unit-or-finer ulp), so the fraction carries one rounding of a number
// in [0, 1], and the error of amin only slides the point along the ray.
__device__ __forceinline__ void axis_walk(float q0, float d, float amin, float amax, int lo, int hi,
                                          float &t, float &D, int &c, int &i0) {
    const float e = fmaf(amin, d, q0), x = fmaf(amax, d, q0);
    int i, ee;
    if (d > 0.f) {
        i = (int)floorf(e);
        ee = (int)ceilf(x) - 1;
    } else if (d < 0.f) {
        i = (int)ceilf(e) - 1;
        ee = (int)floorf(x);
    } else {
        i = (int)floorf(q0);
        ee = i;
    }
    i = min(max(i, lo), hi - 1);
    ee = min(max(ee, lo), hi - 1);
    if (d > 0.f) ee = max(ee, i);
    if (d < 0.f) ee = min(ee, i);
    c = abs(ee - i);
    i0 = i;
    if (d == 0.f) {
        t = kInf;
        D = kInf;
        return;
    }
    D = fabsf(1.0f / d);
    const float f = fminf(fmaxf(fmaf(amin, d, q0 - (float)i), 0.f), 1.f);   // in [0, 1]
    t = (d > 0.f ? 1.f - f : f) * D;   // to the next plane (the exit face if c == 0)
}

// Set up the walk of the ray of pixel (u, v) at view a through the volume box
// with the block axis limited to planes [plo, phi). False if the ray misses.
// With yfast the voxel indices address a copy of the volume stored [z][x][y]
// (y fastest) instead of [z][y][x].
__device__ __forceinline__ bool ray_setup(const DeviceGeom &G, int a, int u, int v, int plo,
                                          int phi, RayWalk &w, bool yfast = false) {
    // ViewRay: p0[3] pu[3] c0[3] cu[3] cv[3] pad; pixel offsets from the detector
    // centre are exact in FP32
    const float4 *p = reinterpret_cast<const float4 *>(G.rays + a);
    const float4 A = __ldg(p + 0), B = __ldg(p + 1), C = __ldg(p + 2), D = __ldg(p + 3);
    const float r[16] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w,
                         C.x, C.y, C.z, C.w, D.x, D.y, D.z, D.w};
    const float fu = (float)u - 0.5f * (float)(G.nu - 1);
    const float fv = (float)v - 0.5f * (float)(G.nv - 1);
    float q0[3], d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        q0[k] = fmaf(fu, r[3 + k], r[k]);
        const float q1 = fmaf(fv, r[12 + k], fmaf(fu, r[9 + k], r[6 + k]));
        d[k] = q1 - q0[k];
    }
    const int lo[3] = {G.axis == 0 ? plo : 0, G.axis == 1 ? plo : 0, G.axis == 2 ? plo : 0};
    const int hi[3] = {G.axis == 0 ? phi : G.nx, G.axis == 1 ? phi : G.ny, G.axis == 2 ? phi : G.nz};
    float amin = 0.f, amax = 1.f;
    int ex = -1;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) ok &= clip_axis(q0[k], d[k], (float)lo[k], (float)hi[k], k, amin, amax, ex);
    // both ray ends lie outside the volume, so a ray that meets the box leaves
    // it through a face (ex >= 0)
    if (!ok || !(amin < amax) || ex < 0) return false;
    int i0[3];
    axis_walk(q0[0], d[0], amin, amax, lo[0], hi[0], w.tx, w.Dx, w.cx, i0[0]);
    axis_walk(q0[1], d[1], amin, amax, lo[1], hi[1], w.ty, w.Dy, w.cy, i0[1]);
    axis_walk(q0[2], d[2], amin, amax, lo[2], hi[2], w.tz, w.Dz, w.cz, i0[2]);
    // parameter of the last interior crossing and of the exit face, each from
    // the entry in one rounding (plane k of an axis lies at t0 + k D)
    {
        float last = 0.f;
        if (w.cx > 0) last = fmaxf(last, fmaf((float)(w.cx - 1), w.Dx, w.tx));
        if (w.cy > 0) last = fmaxf(last, fmaf((float)(w.cy - 1), w.Dy, w.ty));
        if (w.cz > 0) last = fmaxf(last, fmaf((float)(w.cz - 1), w.Dz, w.tz));
        const float face = ex == 0 ? fmaf((float)w.cx, w.Dx, w.tx)
                         : ex == 1 ? fmaf((float)w.cy, w.Dy, w.ty)
                                   : fmaf((float)w.cz, w.Dz, w.tz);
        w.fin = fmaxf(face - last, 0.f);
    }
    w.vmax = (unsigned)(G.nx * G.ny * G.nz - 1);
    // the exit axis's plane after its last interior plane is the exit face
    w.ex = ex;
    w.te = kInf;
    if (ex == 0 && w.cx == 0) { w.te = w.tx; w.tx = kInf; }
    if (ex == 1 && w.cy == 0) { w.te = w.ty; w.ty = kInf; }
    if (ex == 2 && w.cz == 0) { w.te = w.tz; w.tz = kInf; }
    if (w.cx == 0) w.tx = kInf;
    if (w.cy == 0) w.ty = kInf;
    if (w.cz == 0) w.tz = kInf;
    const int strx = yfast ? G.ny : 1, stry = yfast ? 1 : G.nx, strz = G.nx * G.ny;
    w.sx = d[0] > 0.f ? strx : -strx;
    w.sy = d[1] > 0.f ? stry : -stry;
    w.sz = d[2] > 0.f ? strz : -strz;
    w.idx = i0[2] * strz + i0[1] * stry + i0[0] * strx;
    w.n = w.cx + w.cy + w.cz;
    const float lx = d[0] * G.hx, ly = d[1] * G.hy, lz = d[2] * G.hz;
    w.L = sqrtf(fmaf(lx, lx, fmaf(ly, ly, lz * lz)));
    return true;
}

// Visit every voxel of the walk: f(voxel, parameter length of the segment).
// This is the exact form, used where segments are counted against a length
// threshold. Each step takes the nearest interior plane, subtracts the step from the other
// remaining parameters (small numbers, so little rounding) and resets the
// crossed axis to exactly one plane spacing. Only axes with interior planes
// left can step, so the voxel index never leaves the box of entry and exit
// voxels. Ties step x, then y, then z; the tied axis follows with a
// zero-length segment.
template <class F>
__device__ __forceinline__ void ray_walk(RayWalk &w, F &&f) {
    for (int t = 0; t < w.n; ++t) {
        const float s = fminf(w.tx, fminf(w.ty, w.tz));
        f(w.idx, s);
        w.tx -= s;
        w.ty -= s;
        w.tz -= s;
        w.te -= s;
        if (w.tx == 0.f) {
            w.idx += w.sx;
            if (--w.cx > 0) w.tx = w.Dx;
            else { w.tx = kInf; if (w.ex == 0) w.te = w.Dx; }
        } else if (w.ty == 0.f) {
            w.idx += w.sy;
            if (--w.cy > 0) w.ty = w.Dy;
            else { w.ty = kInf; if (w.ex == 1) w.te = w.Dy; }
        } else {
            w.idx += w.sz;
            if (--w.cz > 0) w.tz = w.Dz;
            else { w.tz = kInf; if (w.ex == 2) w.te = w.Dz; }
        }
    }
    f(w.idx, w.te < kInf ? fmaxf(w.te, 0.f) : 0.f);
}

// The same walk for the projector and solver kernels, with about half the
// instructions per step: no per-axis plane counts (a crossed axis always resets
// to one plane spacing), a branch-free choice of the crossed axis, and the last
// segment taken from the set-up (exit face minus last interior crossing).
// Without the counts an axis whose planes are used up could be chosen again,
// but only where its next plane (at or beyond the exit) and a pending interior
// crossing lie within the rounding of the remaining parameters of each other:
// at the very end of the ray, for a sliver of that rounding's length. Voxel
// indices are clamped to the volume, so such a sliver can never address memory
// outside it; FP and BP share this walk, so they stay exact adjoints.
template <class F>
__device__ __forceinline__ void ray_walk_fast(const RayWalk &w, F &&f) {
    float tx = w.tx, ty = w.ty, tz = w.tz;
    int idx = w.idx;
#pragma unroll 4
    for (int t = 0; t < w.n; ++t) {
        const float s = fminf(tx, fminf(ty, tz));
        f((int)min((unsigned)idx, w.vmax), s);
        tx -= s;
        ty -= s;
        tz -= s;
        const bool bx = tx == 0.f;
        const bool by = !bx && ty == 0.f;
        idx += bx ? w.sx : (by ? w.sy : w.sz);
        tx = bx ? w.Dx : tx;
        ty = by ? w.Dy : ty;
        tz = (!bx && !by) ? w.Dz : tz;
    }
    f((int)min((unsigned)idx, w.vmax), w.fin);
}

// Band of view a for column blocks [j0, j1) (entry N of the table is the
// whole volume).
__device__ __forceinline__ Band band_of(const DeviceGeom &G, int a, int j0, int j1) {
    const int stride = G.N + 1;
    if (j0 == 0 && j1 == G.N) return G.bands[(size_t)a * stride + G.N];
    Band b{1 << 30, -1, 1 << 30, -1};
    for (int j = j0; j < j1; ++j) {
        const Band c = G.bands[(size_t)a * stride + j];
        if (c.u0 > c.u1 || c.v0 > c.v1) continue;
        b.u0 = min(b.u0, c.u0);
        b.u1 = max(b.u1, c.u1);
        b.v0 = min(b.v0, c.v0);
        b.v1 = max(b.v1, c.v1);
    }
    return b;
}

// Pixel of this thread inside tile `tile` of band b; false if outside the band.
// 3D: a CTA of 128 threads covers 32 u x 4 v pixels, one warp per detector row:
// the 32 rays of a warp lie side by side across their direction of travel, so
// at equal steps they touch voxels that are neighbours along one axis (the
// fast axis of the layout the solver picks for the view). 2D: 128 consecutive
// bins.
template <bool kThreeD>
__device__ __forceinline__ bool tile_pixel(const Band &b, int tile, int &u, int &v, int &ntiles) {
    constexpr int TU = kThreeD ? kTileU3 : kTileU2;
    constexpr int TV = kThreeD ? kTileV3 : kTileV2;
    if (b.u0 > b.u1 || b.v0 > b.v1) {
        ntiles = 0;
        return false;
    }
    const int ntu = (b.u1 - b.u0 + TU) / TU;
    ntiles = ntu * ((b.v1 - b.v0 + TV) / TV);
    const int tu = tile % ntu, tv = tile / ntu;
    int lu, lv;
    if (kThreeD) {
        lu = threadIdx.x & 31;
        lv = threadIdx.x >> 5;
    } else {
        lu = threadIdx.x;
        lv = 0;
    }
    u = b.u0 + tu * TU + lu;
    v = b.v0 + tv * TV + lv;
    return tile < ntiles && u <= b.u1 && v <= b.v1;
}

}  // namespace bsgd
