// Geometry: validation, ray tables, row/column blocks and detector bands.
//
// Row blocks I_i are sets of whole views and column blocks J_j are slabs of
// whole planes along the block axis (Sec. 2, Eq. 3). Everything here is host
// code in FP64; the per-view ray table is rounded to FP32 once, in voxel units
// relative to the volume's low corner, for the traversal kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "bsgd_internal.h"

namespace bsgd {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }
const char *last_error_cstr() { return g_last_error.c_str(); }

bsgd_status fail(bsgd_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

bsgd_status check_device(const bsgd_geometry *g) {
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BSGD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    if (dev != g->device)
        return fail(BSGD_ERR_INVALID_ARG, "the current CUDA device (" + std::to_string(dev) +
                                              ") is not the geometry's (" + std::to_string(g->device) + ")");
    return BSGD_OK;
}

bsgd_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return BSGD_ERR_CUDA;
}

bsgd_status upload(void **dst, const void *src, size_t bytes) {
    *dst = nullptr;
    if (bytes == 0) return BSGD_OK;
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) {
        *dst = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? BSGD_ERR_OOM : BSGD_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    BSGD_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return BSGD_OK;
}

size_t dtype_size(bsgd_dtype t) { return t == BSGD_F32 ? 4 : 2; }
bool dtype_ok(int t) { return t == BSGD_F32 || t == BSGD_BF16 || t == BSGD_F16; }

namespace {

struct Vec3 {
    double x, y, z;
};

// cos and sin of view angle b. Within 1e-9 rad of a multiple of pi / 2 the
// angle is that multiple exactly: the view's directions are axis-aligned, so a
// ray that lies in a voxel face lies exactly in it, in FP32 as well (double
// cos(pi / 2) is 6e-17, a tilt that would decide which of the face's two voxel
// columns receives the whole ray).
void view_cos_sin(double b, double *c, double *s) {
    const double quarter = 1.5707963267948966;   // pi / 2
    const double k = std::nearbyint(b / quarter);
    if (std::fabs(b - k * quarter) <= 1e-9) {
        const long long m = (((long long)k % 4) + 4) % 4;
        *c = m == 0 ? 1.0 : (m == 2 ? -1.0 : 0.0);
        *s = m == 1 ? 1.0 : (m == 3 ? -1.0 : 0.0);
        return;
    }
    *c = std::cos(b);
    *s = std::sin(b);
}

// Detector coordinates (u, v) of the shadow of point X at view angle b
// (divergent beams): the ray from the source through X meets the detector plane
// at t = dsd / (dso - X . e_r), u = t (X . e_u), v = t X_z.
void shadow(const bsgd_geometry_desc &d, double b, const Vec3 &X, double *u, double *v) {
    double c, s;
    view_cos_sin(b, &c, &s);
    double xu = -s * X.x + c * X.y;
    if (d.kind == BSGD_PAR2D) {
        *u = xu;
        *v = 0.0;
        return;
    }
    double t = d.dsd / (d.dso - (c * X.x + s * X.y));
    *u = t * xu;
    *v = t * X.z;
}

void block_box(const bsgd_geometry *g, int p0, int p1, Vec3 *lo, Vec3 *hi) {
    const bsgd_geometry_desc &d = g->desc;
    lo->x = -0.5 * d.nx * d.dx;
    lo->y = -0.5 * d.ny * d.dy;
    lo->z = -0.5 * d.nz * d.dz;
    hi->x = -lo->x;
    hi->y = -lo->y;
    hi->z = -lo->z;
    if (g->axis == 2) {
        lo->z = -0.5 * d.nz * d.dz + p0 * d.dz;
        hi->z = -0.5 * d.nz * d.dz + p1 * d.dz;
    } else {
        lo->y = -0.5 * d.ny * d.dy + p0 * d.dy;
        hi->y = -0.5 * d.ny * d.dy + p1 * d.dy;
    }
}

// Pixel-centre index range covered by the coordinate interval [lo, hi] on an
// axis of n pixels of size h: k with (k - (n-1)/2) h in [lo, hi].
void pixel_range(double lo, double hi, int n, double h, int margin, int *k0, int *k1) {
    double off = 0.5 * (n - 1);
    double a = std::ceil(lo / h + off) - margin;
    double b = std::floor(hi / h + off) + margin;
    a = std::max(a, 0.0);
    b = std::min(b, (double)(n - 1));
    if (a > b) {
        *k0 = 1;
        *k1 = 0;
        return;
    }
    *k0 = (int)a;
    *k1 = (int)b;
}

// Footprint rectangle of planes [p0, p1) at view a.
void footprint(const bsgd_geometry *g, int a, int p0, int p1, double *umin, double *umax,
               double *vmin, double *vmax) {
    Vec3 lo, hi;
    block_box(g, p0, p1, &lo, &hi);
    *umin = *vmin = 1e300;
    *umax = *vmax = -1e300;
    for (int k = 0; k < 8; ++k) {
        Vec3 X{(k & 1) ? hi.x : lo.x, (k & 2) ? hi.y : lo.y, (k & 4) ? hi.z : lo.z};
        double u, v;
        shadow(g->desc, g->angles[a], X, &u, &v);
        *umin = std::min(*umin, u);
        *umax = std::max(*umax, u);
        *vmin = std::min(*vmin, v);
        *vmax = std::max(*vmax, v);
    }
}

bsgd_status validate(const bsgd_geometry_desc *d, int M, int N) {
    if (!d) return fail(BSGD_ERR_INVALID_ARG, "desc is NULL");
    if (d->kind < BSGD_PAR2D || d->kind > BSGD_CONE3D)
        return fail(BSGD_ERR_INVALID_ARG, "unknown geometry kind");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nu < 1 || d->nv < 1 || d->n_views < 1)
        return fail(BSGD_ERR_INVALID_ARG, "sizes must be >= 1");
    if (!(d->dx > 0) || !(d->dy > 0) || !(d->dz > 0) || !(d->du > 0) || !(d->dv > 0))
        return fail(BSGD_ERR_INVALID_ARG, "voxel and pixel sizes must be > 0");
    // every ray parameter must stay finite: the traversal's step counts rely on it
    for (double v : {d->dx, d->dy, d->dz, d->du, d->dv, d->dso, d->dsd})
        if (!std::isfinite(v)) return fail(BSGD_ERR_INVALID_ARG, "sizes and distances must be finite");
    if (d->kind != BSGD_CONE3D && (d->nz != 1 || d->nv != 1))
        return fail(BSGD_ERR_INVALID_ARG, "2D geometries need nz == nv == 1");
    if ((double)d->nx * d->ny * d->nz > 2147483647.0)
        return fail(BSGD_ERR_INVALID_ARG, "more than 2^31-1 voxels");
    if ((double)d->n_views * d->nu * d->nv > 2147483647.0)
        return fail(BSGD_ERR_INVALID_ARG, "more than 2^31-1 rays");
    if (d->kind != BSGD_PAR2D) {
        if (!(d->dso > 0) || !(d->dsd > d->dso))
            return fail(BSGD_ERR_INVALID_ARG, "need 0 < dso < dsd");
        double hx = 0.5 * d->nx * d->dx, hy = 0.5 * d->ny * d->dy;
        if (std::sqrt(hx * hx + hy * hy) >= d->dso)
            return fail(BSGD_ERR_INVALID_ARG, "volume reaches the source circle");
        // every ray must leave the volume before the detector
        if (std::sqrt(hx * hx + hy * hy) >= d->dsd - d->dso)
            return fail(BSGD_ERR_INVALID_ARG, "volume reaches the detector plane");
    }
    int planes = d->nz > 1 ? d->nz : d->ny;
    if (M < 1 || M > d->n_views) return fail(BSGD_ERR_INVALID_ARG, "need 1 <= M <= n_views");
    if (N < 1 || N > planes)
        return fail(BSGD_ERR_INVALID_ARG, "need 1 <= N <= planes along the block axis");
    if (d->angles)
        for (int a = 0; a < d->n_views; ++a)
            if (!std::isfinite(d->angles[a]))
                return fail(BSGD_ERR_INVALID_ARG, "angles must be finite");
    if (d->view_block) {
        std::vector<int> cnt(M, 0);
        for (int a = 0; a < d->n_views; ++a) {
            if (d->view_block[a] < 0 || d->view_block[a] >= M)
                return fail(BSGD_ERR_INVALID_ARG, "view_block id out of range");
            cnt[d->view_block[a]]++;
        }
        for (int i = 0; i < M; ++i)
            if (!cnt[i]) return fail(BSGD_ERR_INVALID_ARG, "a row block has no views");
    }
    return BSGD_OK;
}

}  // namespace

bsgd_status validate_desc(const bsgd_geometry_desc *d, int M, int N) { return validate(d, M, N); }

int tiles_for(const bsgd_geometry *g, const std::vector<int> &views, int j0, int j1, int tu,
              int tv) {
    int best = 0;
    const int stride = g->N + 1;
    for (int a : views) {
        Band b{1 << 30, -1, 1 << 30, -1};
        if (j0 == 0 && j1 == g->N) {
            b = g->bands[(size_t)a * stride + g->N];
        } else {
            for (int j = j0; j < j1; ++j) {
                const Band &c = g->bands[(size_t)a * stride + j];
                if (c.u0 > c.u1 || c.v0 > c.v1) continue;
                b.u0 = std::min(b.u0, c.u0);
                b.u1 = std::max(b.u1, c.u1);
                b.v0 = std::min(b.v0, c.v0);
                b.v1 = std::max(b.v1, c.v1);
            }
        }
        if (b.u0 > b.u1 || b.v0 > b.v1) continue;
        int t = ((b.u1 - b.u0 + tu) / tu) * ((b.v1 - b.v0 + tv) / tv);
        best = std::max(best, t);
    }
    return best;
}

}  // namespace bsgd

using namespace bsgd;

static void free_geometry(bsgd_geometry *g) {
    cudaFree(g->d_rays);
    cudaFree(g->d_bands);
    cudaFree(g->d_block_views);
    cudaFree(g->d_block_nviews);
    cudaFree(g->d_plane_start);
    cudaFree(g->d_view_block);
    cudaFree(g->d_view_yfast);
    cudaFree(g->d_zoff);
    for (int k = 0; k < 5; ++k) {
        cudaFree(g->d_counts[k]);
        cudaFree(g->d_cw[k]);
    }
    delete g;
}

namespace bsgd {
bsgd_status build_host_tables(const bsgd_geometry_desc *desc, int M, int N, bsgd_geometry *g) {
    BSGD_TRY(validate(desc, M, N));
    const bsgd_geometry_desc &d = *desc;
    g->desc = d;
    g->M = M;
    g->N = N;
    g->axis = d.nz > 1 ? 2 : 1;
    g->n_planes = g->axis == 2 ? d.nz : d.ny;
    g->angles.resize(d.n_views);
    const double span = d.kind == BSGD_PAR2D ? M_PI : 2.0 * M_PI;
    for (int a = 0; a < d.n_views; ++a)
        g->angles[a] = d.angles ? d.angles[a] : a * (span / d.n_views);
    g->view_block.resize(d.n_views);
    for (int a = 0; a < d.n_views; ++a) g->view_block[a] = d.view_block ? d.view_block[a] : a % M;
    g->desc.angles = g->angles.data();
    g->desc.view_block = g->view_block.data();

    g->plane_start.resize(N + 1);
    for (int j = 0; j <= N; ++j) g->plane_start[j] = (int)(((int64_t)j * g->n_planes) / N);
    g->block_views.assign(M, {});
    for (int a = 0; a < d.n_views; ++a) g->block_views[g->view_block[a]].push_back(a);
    g->max_views = 0;
    for (auto &bv : g->block_views) g->max_views = std::max(g->max_views, (int)bv.size());

    // ---- ray table (voxel units, origin at the volume's low corner)
    const double lo[3] = {-0.5 * d.nx * d.dx, -0.5 * d.ny * d.dy, -0.5 * d.nz * d.dz};
    const double h[3] = {d.dx, d.dy, d.dz};
    g->rays.resize(d.n_views);
    // Rays are addressed by the pixel's offset from the detector centre,
    // (u - (nu-1)/2, v - (nv-1)/2), which FP32 holds exactly.
    for (int a = 0; a < d.n_views; ++a) {
        double c, s;
        view_cos_sin(g->angles[a], &c, &s);
        const double er[3] = {c, s, 0.0}, eu[3] = {-s, c, 0.0}, ev[3] = {0.0, 0.0, 1.0};
        double p0[3], pu[3], c0[3], cu[3], cv[3];
        if (d.kind == BSGD_PAR2D) {
            // a segment through the bin centre, long enough to cross the box
            double R = std::sqrt(lo[0] * lo[0] + lo[1] * lo[1] + lo[2] * lo[2]) + 1.0;
            for (int k = 0; k < 3; ++k) {
                p0[k] = -R * er[k];
                c0[k] = R * er[k];
                pu[k] = cu[k] = d.du * eu[k];
                cv[k] = 0.0;
            }
        } else {
            const double back = d.dsd - d.dso;
            for (int k = 0; k < 3; ++k) {
                p0[k] = d.dso * er[k];
                pu[k] = 0.0;
                c0[k] = -back * er[k];
                cu[k] = d.du * eu[k];
                cv[k] = d.dv * ev[k];
            }
        }
        ViewRay &R = g->rays[a];
        for (int k = 0; k < 3; ++k) {
            R.p0[k] = (float)((p0[k] - lo[k]) / h[k]);
            R.pu[k] = (float)(pu[k] / h[k]);
            R.c0[k] = (float)((c0[k] - lo[k]) / h[k]);
            R.cu[k] = (float)(cu[k] / h[k]);
            R.cv[k] = (float)(cv[k] / h[k]);
        }
        R.pad = 0.f;
    }

    // ---- detector bands of every (view, column block) and of the whole volume
    const int stride = N + 1;
    g->bands.resize((size_t)d.n_views * stride);
    for (int a = 0; a < d.n_views; ++a) {
        for (int j = 0; j <= N; ++j) {
            int p0 = j < N ? g->plane_start[j] : 0, p1 = j < N ? g->plane_start[j + 1] : g->n_planes;
            double umin, umax, vmin, vmax;
            footprint(g, a, p0, p1, &umin, &umax, &vmin, &vmax);
            Band b;
            pixel_range(umin, umax, d.nu, d.du, 1, &b.u0, &b.u1);
            if (d.nv == 1) {
                b.v0 = b.v1 = 0;
            } else {
                pixel_range(vmin, vmax, d.nv, d.dv, 1, &b.v0, &b.v1);
            }
            g->bands[(size_t)a * stride + j] = b;
        }
    }
    // exact v-band R_ij (no margin): rows whose residual weights pair (i, j)
    g->wband.assign((size_t)M * N * 2, 0);
    for (int i = 0; i < M; ++i) {
        for (int j = 0; j < N; ++j) {
            int lo_v = d.nv, hi_v = -1;
            if (d.nv == 1) {
                lo_v = hi_v = 0;
            } else {
                for (int a : g->block_views[i]) {
                    double umin, umax, vmin, vmax;
                    footprint(g, a, g->plane_start[j], g->plane_start[j + 1], &umin, &umax, &vmin,
                              &vmax);
                    int k0, k1;
                    pixel_range(vmin, vmax, d.nv, d.dv, 0, &k0, &k1);
                    if (k0 <= k1) {
                        lo_v = std::min(lo_v, k0);
                        hi_v = std::max(hi_v, k1);
                    }
                }
            }
            g->wband[((size_t)i * N + j) * 2 + 0] = lo_v;
            g->wband[((size_t)i * N + j) * 2 + 1] = hi_v;
        }
    }

    // ---- compact band storage: block j's rows of view a, band by band
    g->zoff.assign((size_t)N * d.n_views, 0);
    int64_t off = 0;
    for (int j = 0; j < N; ++j) {
        for (int a = 0; a < d.n_views; ++a) {
            g->zoff[(size_t)j * d.n_views + a] = off;
            const Band &b = g->bands[(size_t)a * stride + j];
            if (b.u0 <= b.u1 && b.v0 <= b.v1) off += (int64_t)(b.u1 - b.u0 + 1) * (b.v1 - b.v0 + 1);
        }
    }
    g->zlen = off;
    return BSGD_OK;
}
}  // namespace bsgd

extern "C" bsgd_status bsgd_geometry_create(const bsgd_geometry_desc *desc, int M, int N,
                                            bsgd_geometry **out) {
    if (!out) return fail(BSGD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    bsgd_geometry *g = new (std::nothrow) bsgd_geometry();
    if (!g) return fail(BSGD_ERR_OOM, "host allocation failed");
    {
        bsgd_status st = build_host_tables(desc, M, N, g);
        if (st) {
            delete g;
            return st;
        }
    }
    const bsgd_geometry_desc &d = *desc;

    // ---- upload
    std::vector<int> bv((size_t)M * g->max_views, -1), bn(M);
    for (int i = 0; i < M; ++i) {
        bn[i] = (int)g->block_views[i].size();
        for (int k = 0; k < bn[i]; ++k) bv[(size_t)i * g->max_views + k] = g->block_views[i][k];
    }
    // views whose rays run mostly along x (|cos| > |sin| of the view angle)
    // use the y-fastest copies of the solver state (volumes only)
    std::vector<unsigned char> yfast(d.n_views, 0);
    for (int a = 0; a < d.n_views && d.nz > 1; ++a) {
        double c, s;
        view_cos_sin(g->angles[a], &c, &s);
        yfast[a] = std::fabs(c) > std::fabs(s) ? 1 : 0;
    }
    g->view_yfast = yfast;
    bsgd_status st = BSGD_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    g->device = dev;
    if ((st = upload((void **)&g->d_rays, g->rays.data(), g->rays.size() * sizeof(ViewRay))) ||
        (st = upload((void **)&g->d_bands, g->bands.data(), g->bands.size() * sizeof(Band))) ||
        (st = upload((void **)&g->d_block_views, bv.data(), bv.size() * sizeof(int))) ||
        (st = upload((void **)&g->d_block_nviews, bn.data(), bn.size() * sizeof(int))) ||
        (st = upload((void **)&g->d_plane_start, g->plane_start.data(), (N + 1) * sizeof(int))) ||
        (st = upload((void **)&g->d_view_block, g->view_block.data(),
                     g->view_block.size() * sizeof(int))) ||
        (st = upload((void **)&g->d_view_yfast, yfast.data(), yfast.size())) ||
        (st = upload((void **)&g->d_zoff, g->zoff.data(), g->zoff.size() * sizeof(int64_t)))) {
        free_geometry(g);
        return st;
    }
    DeviceGeom &dg = g->dg;
    dg.rays = g->d_rays;
    dg.bands = g->d_bands;
    dg.block_views = g->d_block_views;
    dg.block_nviews = g->d_block_nviews;
    dg.plane_start = g->d_plane_start;
    dg.view_block = g->d_view_block;
    dg.view_yfast = g->d_view_yfast;
    dg.zoff = g->d_zoff;
    dg.zlen = g->zlen;
    dg.nx = d.nx;
    dg.ny = d.ny;
    dg.nz = d.nz;
    dg.hx = (float)d.dx;
    dg.hy = (float)d.dy;
    dg.hz = (float)d.dz;
    dg.nu = d.nu;
    dg.nv = d.nv;
    dg.n_views = d.n_views;
    dg.M = M;
    dg.N = N;
    dg.axis = g->axis;
    dg.max_views = g->max_views;
    dg.n_rows = g->n_rows();
    dg.n_cols = g->n_cols();
    dg.plane_stride = g->axis == 2 ? d.nx * d.ny : d.nx;
    *out = g;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_geometry_destroy(bsgd_geometry *g) {
    if (!g) return fail(BSGD_ERR_INVALID_ARG, "geometry is NULL");
    free_geometry(g);
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_geometry_get_info(const bsgd_geometry *g, bsgd_geometry_info *out) {
    if (!g || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    out->n_rows = g->n_rows();
    out->n_cols = g->n_cols();
    out->M = g->M;
    out->N = g->N;
    out->block_axis = g->axis;
    out->max_views_per_block = g->max_views;
    int64_t m = 0;
    for (int j = 0; j < g->N; ++j) m = std::max(m, g->block_cols(j));
    out->max_block_cols = m;
    out->compact_rows = g->zlen;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_geometry_pair_rays(const bsgd_geometry *g, int i, int j, int64_t *out) {
    if (!g || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (i < 0 || i >= g->M || j < 0 || j >= g->N) return fail(BSGD_ERR_INVALID_ARG, "block id out of range");
    int64_t n = 0;
    for (int a : g->block_views[i]) {
        const Band &b = g->bands[(size_t)a * (g->N + 1) + j];
        if (b.u0 <= b.u1 && b.v0 <= b.v1) n += (int64_t)(b.u1 - b.u0 + 1) * (b.v1 - b.v0 + 1);
    }
    *out = n;
    return BSGD_OK;
}
