// BSGD solver state and the per-iteration kernels other than the projector:
// block sampling, residual recomputation, the block step, FP64 residual-norm
// tables and the power-iteration step size.
//
// One iteration (Algorithm 1; Algorithm 2 with sub-detector cells):
//   sample_kernel     picks the pairs (i, j) (and cells) on the device
//   fp_solve_kernel   z^j_R = A_R^J x_J, r_R = y_R - sum_j z^j_R   (siddon.cu)
//   residual_kernel   only when several column blocks share a row block
//   bp_solve_kernel   g_J += (A_R^J)^T (r_R - r~^J_R), r~^J_R = r_R (siddon.cu)
//   update_kernel     x_J += mu g_J
// The snapshot r~^J equals keeping Algorithm 1's memory g-hat^i: it stores the
// residual the last BP of (i, J) used, so the BP of the change replaces
// g-hat^i_J by the new one exactly.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "siddon_device.cuh"

namespace bsgd {

// ---------------------------------------------------------------------------
// SplitMix64 counter spec (Steele, Lea and Flood 2014): draw number
// n = it * 2^20 + lane + 1 of the generator seeded with `seed` is
// mix(seed + n * 0x9E3779B97F4A7C15); u = (draw >> 11) * 2^-53.

constexpr int kLaneRows = 0, kLaneCols = 256, kLanePair = 1024, kLaneCells = 2048;
constexpr double kResidualFloor = 1e-9;
constexpr double kCellFloor = 1e-12;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline double draw_u(uint64_t seed, int64_t it, int lane) {
    const uint64_t n = ((uint64_t)it << 20) + (uint64_t)lane + 1ull;
    return (double)(mix64(seed + n * 0x9E3779B97F4A7C15ull) >> 11) * (1.0 / 9007199254740992.0);
}

// smallest index whose running FP64 sum exceeds u * total
__device__ inline int pick_weighted(double u, const double *w, int n, int stride) {
    double tot = 0.0;
    for (int k = 0; k < n; ++k) tot += w[k * stride];
    const double c = u * tot;
    double acc = 0.0;
    int last = 0;
    for (int k = 0; k < n; ++k) {
        acc += w[k * stride];
        if (w[k * stride] > 0.0) last = k;
        if (acc > c) return k;
    }
    return last;
}

constexpr int kSampleThreads = 256;
constexpr int kMaxSampleBlocks = 1024;
constexpr int kMaxResidualPairs = 1024;
constexpr int kSampleSmemS = 2048;     // residual-table entries staged in shared memory

// One iteration's draw (Algorithm 1's selection step; Algorithm 2's per-view
// cells), executed by one CTA of kSampleThreads threads. Writes the work list,
// the chosen cells, the trace entry and the update counter, then advances the
// iteration counter.
// Residual-pair weights W_k = sum over the pair's detector rows of S[i][v] for
// the pairs k0 <= k < k1, one warp per pair (lanes over rows in a fixed order,
// then a fixed shuffle tree): the same sums whichever CTA computes them.
__device__ void pair_weights(const SampleArgs &A, const double *S, int k0, int k1, double *out) {
    const DeviceGeom &G = A.G;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int k = k0 + warp; k < k1; k += nwarps) {
        const int lo = A.wband[2 * k], hi = A.wband[2 * k + 1];
        const int i = k / G.N;
        double w = 0.0;
        for (int v = lo + lane; v <= hi; v += 32) w += S[(size_t)i * G.nv + v];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) out[k] = w;
    }
}

__device__ void sample_body(const SampleArgs &A, const double *pre_w = nullptr) {
    // one buffer, two uses: the uniform draw's permutations, or the residual
    // table (staged with one parallel load: the draw is a latency chain) and
    // the pair weights
    __shared__ double s_buf[kSampleSmemS + kMaxResidualPairs];
    static_assert(2 * kMaxSampleBlocks * sizeof(int) <= sizeof(s_buf), "permutation buffers");
    int *s_rows = reinterpret_cast<int *>(s_buf);
    int *s_cols = s_rows + kMaxSampleBlocks;
    double *s_S = s_buf;
    double *s_w = s_buf + kSampleSmemS;
    __shared__ int s_np;
    __shared__ int s_pi[kMaxPairs], s_pj[kMaxPairs];
    __shared__ unsigned long long s_upd;
    const DeviceGeom &G = A.G;
    const int64_t it = A.it >= 0 ? A.it : *A.iter;
    const int tid = threadIdx.x;
    const bool replay = A.replay && it >= A.replay_start && it - A.replay_start < A.replay_n;
    const int32_t *rep = replay ? A.replay + (it - A.replay_start) * A.stride : nullptr;
    if (tid == 0) s_upd = 0ull;

    if (replay) {
        if (tid == 0) {
            s_np = rep[0];
            for (int p = 0; p < s_np; ++p) {
                s_pi[p] = rep[1 + 2 * p];
                s_pj[p] = rep[2 + 2 * p];
            }
        }
    } else if (A.pairs_mode == BSGD_PAIRS_UNIFORM) {
        if (tid == 0) {
            for (int k = 0; k < G.M; ++k) s_rows[k] = k;
            for (int t = 0; t < A.kM; ++t) {  // partial Fisher-Yates
                const int idx = t + (int)(draw_u(A.seed, it, kLaneRows + t) * (G.M - t));
                const int tmp = s_rows[t]; s_rows[t] = s_rows[idx]; s_rows[idx] = tmp;
            }
            for (int k = 0; k < G.N; ++k) s_cols[k] = k;
            for (int t = 0; t < A.kN; ++t) {
                const int idx = t + (int)(draw_u(A.seed, it, kLaneCols + t) * (G.N - t));
                const int tmp = s_cols[t]; s_cols[t] = s_cols[idx]; s_cols[idx] = tmp;
            }
            // sort the chosen prefixes (insertion sort; k is small)
            for (int a = 1; a < A.kM; ++a)
                for (int b = a; b > 0 && s_rows[b - 1] > s_rows[b]; --b) {
                    const int t = s_rows[b]; s_rows[b] = s_rows[b - 1]; s_rows[b - 1] = t;
                }
            for (int a = 1; a < A.kN; ++a)
                for (int b = a; b > 0 && s_cols[b - 1] > s_cols[b]; --b) {
                    const int t = s_cols[b]; s_cols[b] = s_cols[b - 1]; s_cols[b - 1] = t;
                }
            int np = 0;
            for (int a = 0; a < A.kM; ++a)
                for (int b = 0; b < A.kN; ++b) {
                    s_pi[np] = s_rows[a];
                    s_pj[np] = s_cols[b];
                    ++np;
                }
            s_np = np;
        }
    } else if (pre_w) {  // residual-weighted pair, weights computed by other CTAs
        const int MN = G.M * G.N;
        const int warp = tid >> 5, lane = tid & 31;
        for (int k = tid; k < MN; k += blockDim.x) s_w[k] = __ldcg(pre_w + k);
        __syncthreads();
        if (warp == 0) {
            double t = 0.0;
            for (int k = lane; k < MN; k += 32) t += s_w[k];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            const double fl = kResidualFloor * t / MN + 1e-300;
            double carry = 0.0;
            for (int b = 0; b < MN; b += 32) {
                double v = b + lane < MN ? s_w[b + lane] + fl : 0.0;
                for (int o = 1; o < 32; o <<= 1) {
                    const double n = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += n;
                }
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
            const double c = draw_u(A.seed, it, kLanePair) * carry;
            int pick = -1;
            carry = 0.0;
            for (int b = 0; b < MN && pick < 0; b += 32) {
                double v = b + lane < MN ? s_w[b + lane] + fl : 0.0;
                for (int o = 1; o < 32; o <<= 1) {
                    const double n = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += n;
                }
                v += carry;
                const unsigned hit = __ballot_sync(0xffffffffu, b + lane < MN && v > c);
                if (hit) pick = b + __ffs(hit) - 1;
                carry = __shfl_sync(0xffffffffu, v, 31);
            }
            if (pick < 0) pick = MN - 1;
            if (lane == 0) {
                s_np = 1;
                s_pi[0] = pick / G.N;
                s_pj[0] = pick % G.N;
            }
        }
    } else {  // residual-weighted pair: W_ij = sum_{v in R_ij} S[i][v] + floor
        const int MN = G.M * G.N;
        const int nS = G.M * G.nv;
        const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
        const bool staged = nS <= kSampleSmemS;
        // the first batch of band limits is fetched with the staging loads
        const int kl0 = warp + lane * nwarps;
        const int lo0 = kl0 < MN ? A.wband[2 * kl0] : 0;
        const int hi0 = kl0 < MN ? A.wband[2 * kl0 + 1] : -1;
        if (staged) {
#pragma unroll 8
            for (int k = tid; k < nS; k += blockDim.x) s_S[k] = A.S[k];
        }
        __syncthreads();
        const double *S = staged ? s_S : A.S;
        // a warp per pair, its lanes over the pair's detector rows (fixed
        // order); a batch of 32 pairs' band limits is fetched in one load per
        // lane and handed round by shuffles
        for (int k0 = warp; k0 < MN; k0 += 32 * nwarps) {
            const int kl = k0 + lane * nwarps;
            const int lo_l = k0 == warp ? lo0 : (kl < MN ? A.wband[2 * kl] : 0);
            const int hi_l = k0 == warp ? hi0 : (kl < MN ? A.wband[2 * kl + 1] : -1);
            for (int t = 0; t < 32 && k0 + t * nwarps < MN; ++t) {
                const int k = k0 + t * nwarps;
                const int lo = __shfl_sync(0xffffffffu, lo_l, t), hi = __shfl_sync(0xffffffffu, hi_l, t);
                const int i = k / G.N;
                double w = 0.0;
                for (int v = lo + lane; v <= hi; v += 32) w += S[(size_t)i * G.nv + v];
                for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                if (lane == 0) s_w[k] = w;
            }
        }
        __syncthreads();
        if (warp == 0) {
            // floor, then the draw: the smallest k whose running sum exceeds
            // u * total, with the running sums from a warp scan in chunks of 32
            double t = 0.0;
            for (int k = lane; k < MN; k += 32) t += s_w[k];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            const double fl = kResidualFloor * t / MN + 1e-300;
            double carry = 0.0;
            for (int b = 0; b < MN; b += 32) {            // pass 1: the total
                double v = b + lane < MN ? s_w[b + lane] + fl : 0.0;
                for (int o = 1; o < 32; o <<= 1) {
                    const double n = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += n;
                }
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
            const double c = draw_u(A.seed, it, kLanePair) * carry;
            int pick = -1;
            carry = 0.0;
            for (int b = 0; b < MN && pick < 0; b += 32) {   // pass 2: the first crossing
                double v = b + lane < MN ? s_w[b + lane] + fl : 0.0;
                for (int o = 1; o < 32; o <<= 1) {
                    const double n = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += n;
                }
                v += carry;
                const unsigned hit = __ballot_sync(0xffffffffu, b + lane < MN && v > c);
                if (hit) pick = b + __ffs(hit) - 1;
                carry = __shfl_sync(0xffffffffu, v, 31);
            }
            if (pick < 0) pick = MN - 1;   // rounding left c at the total: the last pair
            if (lane == 0) {
                s_np = 1;
                s_pi[0] = pick / G.N;
                s_pj[0] = pick % G.N;
            }
        }
    }
    __syncthreads();
    const int np = s_np;
    // cells: one per view of each pair's row block; voxel-ray updates of the
    // chosen rows (FP + BP) summed in parallel (whole views: one table entry
    // per pair)
    unsigned long long upd = 0;
    const bool whole = A.cells_mode == BSGD_CELLS_NONE && A.pair_upd != nullptr;
    if (whole && tid == 0)
        for (int p = 0; p < np; ++p) upd += A.pair_upd[s_pi[p] * G.N + s_pj[p]];
    for (int q = tid; q < np * G.max_views; q += blockDim.x) {
        if (whole) {
            A.cells[q] = -1;
            continue;
        }
        const int p = q / G.max_views, k = q % G.max_views;
        const int i = s_pi[p], j = s_pj[p];
        const int nvb = G.block_nviews[i];
        int c = -1;
        if (k < nvb) {
            const int a = G.block_views[i * G.max_views + k];
            if (A.cells_mode != BSGD_CELLS_NONE) {
                if (replay) {
                    c = rep[1 + 2 * np + p * G.max_views + k];
                } else {
                    const double u = draw_u(A.seed, it, kLaneCells + p * nvb + k);
                    if (A.cells_mode == BSGD_CELLS_UNIFORM)
                        c = min((int)(u * A.n_cells), A.n_cells - 1);
                    else
                        c = pick_weighted(u, A.cw + ((size_t)j * G.n_views + a) * A.n_cells,
                                          A.n_cells, 1);
                }
            }
            const unsigned long long *cn = A.counts + ((size_t)j * G.n_views + a) * A.n_cells;
            if (c >= 0) upd += cn[c];
            else for (int s = 0; s < A.n_cells; ++s) upd += cn[s];
        }
        A.cells[p * G.max_views + k] = c;
    }
    for (int o = 16; o > 0; o >>= 1) upd += __shfl_xor_sync(0xffffffffu, upd, o);
    if ((tid & 31) == 0 && upd) atomicAdd(&s_upd, upd);
    __syncthreads();
    if (tid == 0) {
        Work &W = *A.work;
        W.n_pairs = np;
        int nc = 0, nr = 0;
        for (int p = 0; p < np; ++p) {
            W.pair_i[p] = s_pi[p];
            W.pair_j[p] = s_pj[p];
            bool seen = false;
            for (int t = 0; t < nc; ++t) seen |= W.cols[t] == s_pj[p];
            if (!seen) W.cols[nc++] = s_pj[p];
            seen = false;
            for (int t = 0; t < nr; ++t) seen |= W.rows[t] == s_pi[p];
            if (!seen) W.rows[nr++] = s_pi[p];
        }
        W.n_cols = nc;
        W.n_rows = nr;
        atomicAdd(A.updates, 2ull * s_upd);
        if (A.trace && it < A.trace_cap) {
            int32_t *t = A.trace + it * A.stride;
            t[0] = np;
            for (int p = 0; p < np; ++p) {
                t[1 + 2 * p] = s_pi[p];
                t[2 + 2 * p] = s_pj[p];
            }
        }
    }
    if (A.trace && it < A.trace_cap) {
        int32_t *t = A.trace + it * A.stride;
        for (int q = tid; q < np * G.max_views; q += blockDim.x) t[1 + 2 * np + q] = A.cells[q];
        for (int q = 1 + 2 * np + np * G.max_views + tid; q < A.stride; q += blockDim.x) t[q] = -1;
    }
    __syncthreads();
    if (tid == 0) *A.iter = it + 1;
}

__global__ void __launch_bounds__(kSampleThreads) sample_kernel(const SampleArgs A) { sample_body(A); }

// pair_upd[i][j] = voxel-ray updates of every whole view of row block i in
// column block j (the cell counts summed).
__global__ void pair_updates_kernel(const DeviceGeom G, const unsigned long long *__restrict__ counts,
                                    int n_cells, unsigned long long *__restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= G.M * G.N) return;
    const int i = q / G.N, j = q % G.N;
    unsigned long long t = 0;
    for (int k = 0; k < G.block_nviews[i]; ++k) {
        const unsigned long long *cn =
            counts + ((size_t)j * G.n_views + G.block_views[i * G.max_views + k]) * n_cells;
        for (int c = 0; c < n_cells; ++c) t += cn[c];
    }
    out[q] = t;
}

// r = y - sum_j z^j over the rows of the selected row blocks that the
// iteration's FPs changed (the union of the selected column blocks' bands in
// each view), used when several column blocks of one row block are selected
// so the FPs cannot update r themselves; with the FP64 row-block residual sums,
// reduced over the CTA into one atomic per detector row. A CTA covers
// kResRows detector rows of one view.
constexpr int kResRows = 4;

// Bounding box, at view a, of the bands of the iteration's column blocks: the
// rows whose z^j changed (the residual pass and the sharded exchange cover it).
__device__ __forceinline__ Band union_band(const DeviceGeom &G, const Work &W, int a) {
    Band b{1 << 30, -1, 1 << 30, -1};
    for (int c = 0; c < W.n_cols; ++c) {
        const Band q = G.bands[(size_t)a * (G.N + 1) + W.cols[c]];
        if (q.u0 > q.u1 || q.v0 > q.v1) continue;
        b.u0 = min(b.u0, q.u0);
        b.u1 = max(b.u1, q.u1);
        b.v0 = min(b.v0, q.v0);
        b.v1 = max(b.v1, q.v1);
    }
    return b;
}

template <typename T>
__global__ void __launch_bounds__(256) residual_kernel(const DeviceGeom G, const SolveDev S) {
    const Work &W = *S.work;
    const int rb = blockIdx.z;
    if (rb >= W.n_rows) return;
    const int i = W.rows[rb];
    const int slot = blockIdx.y;
    if (slot >= G.block_nviews[i]) return;
    const int a = G.block_views[i * G.max_views + slot];
    const Band b = union_band(G, W, a);
    const int vbeg = b.v0 + blockIdx.x * kResRows;
    if (b.u0 > b.u1 || vbeg > b.v1) return;
    const T *y = reinterpret_cast<const T *>(S.y);
    const T *z = reinterpret_cast<const T *>(S.z);
    T *r = reinterpret_cast<T *>(S.r);
    __shared__ double sh[8];
    for (int v = vbeg; v < vbeg + kResRows && v <= b.v1; ++v) {
        const int64_t base = ((int64_t)a * G.nv + v) * G.nu;
        double dn = 0.0;
        for (int u = b.u0 + threadIdx.x; u <= b.u1; u += blockDim.x) {
            const int64_t row = base + u;
            float zs = 0.f;
            for (int jj = 0; jj < G.N; ++jj) {   // z^jj is 0 outside block jj's band
                bool in;
                const int64_t kz = zslot(G, jj, a, u, v, in);
                if (in) zs += ldv(z + kz);
            }
            const float rn = rnd(ldf(y + row) - zs, r);
            const float ro = ldv(r + row);
            if (rn != ro) {
                stf(r + row, rn);
                dn += (double)rn * rn - (double)ro * ro;
            }
        }
        for (int o = 16; o > 0; o >>= 1) dn += __shfl_xor_sync(0xffffffffu, dn, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dn;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
            if (t != 0.0) atomicAdd(S.S + (size_t)i * G.nv + v, t);
        }
    }
}

// Owner-computes sharding (one process per device, each owning some column
// blocks): the exchange buffer holds, for every row of the union band in each
// view of each drawn row block, this process's part sum_{owned j} z^j of
// sum_j z^j. The processes sum their buffers (one all-reduce), then each forms
// r = y - sum_j z^j from the total. Layout: [row-block slot][view slot][v][u].
__device__ __forceinline__ int64_t xchg_index(const DeviceGeom &G, int rb, int slot, int v, int u) {
    return (((int64_t)rb * G.max_views + slot) * G.nv + v) * G.nu + u;
}

template <typename T>
__global__ void __launch_bounds__(256) shard_partial_kernel(const DeviceGeom G, const SolveDev S,
                                                            float *__restrict__ xchg) {
    const Work &W = *S.work;
    const int rb = blockIdx.z;
    if (rb >= W.n_rows) return;
    const int i = W.rows[rb], slot = blockIdx.y;
    if (slot >= G.block_nviews[i]) return;
    const int a = G.block_views[i * G.max_views + slot];
    const Band b = union_band(G, W, a);
    const int vbeg = b.v0 + blockIdx.x * kResRows;
    if (b.u0 > b.u1 || vbeg > b.v1) return;
    const T *z = reinterpret_cast<const T *>(S.z);
    for (int v = vbeg; v < vbeg + kResRows && v <= b.v1; ++v)
        for (int u = b.u0 + threadIdx.x; u <= b.u1; u += blockDim.x) {
            float zs = 0.f;
            for (int jj = 0; jj < G.N; ++jj) {
                if (!S.owned[jj]) continue;
                bool in;
                const int64_t kz = zslot(G, jj, a, u, v, in);
                if (in) zs += ldv(z + kz);
            }
            xchg[xchg_index(G, rb, slot, v, u)] = zs;
        }
}

// r = y - (the all-reduced sum of z^j) over the same rows, with the FP64
// residual table updated by the change of r^2.
template <typename T>
__global__ void __launch_bounds__(256) shard_residual_kernel(const DeviceGeom G, const SolveDev S,
                                                             const float *__restrict__ xchg) {
    const Work &W = *S.work;
    const int rb = blockIdx.z;
    if (rb >= W.n_rows) return;
    const int i = W.rows[rb], slot = blockIdx.y;
    if (slot >= G.block_nviews[i]) return;
    const int a = G.block_views[i * G.max_views + slot];
    const Band b = union_band(G, W, a);
    const int vbeg = b.v0 + blockIdx.x * kResRows;
    if (b.u0 > b.u1 || vbeg > b.v1) return;
    const T *y = reinterpret_cast<const T *>(S.y);
    T *r = reinterpret_cast<T *>(S.r);
    __shared__ double sh[8];
    for (int v = vbeg; v < vbeg + kResRows && v <= b.v1; ++v) {
        const int64_t base = ((int64_t)a * G.nv + v) * G.nu;
        double dn = 0.0;
        for (int u = b.u0 + threadIdx.x; u <= b.u1; u += blockDim.x) {
            const int64_t row = base + u;
            const float rn = rnd(ldf(y + row) - xchg[xchg_index(G, rb, slot, v, u)], r);
            const float ro = ldv(r + row);
            if (rn != ro) {
                stf(r + row, rn);
                dn += (double)rn * rn - (double)ro * ro;
            }
        }
        for (int o = 16; o > 0; o >>= 1) dn += __shfl_xor_sync(0xffffffffu, dn, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dn;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
            if (t != 0.0) atomicAdd(S.S + (size_t)i * G.nv + v, t);
        }
    }
}

// x_J += mu g_J for the selected column blocks. With 16-bit storage the
// state keeps a low-order term xlo of the same type (compensated storage): the
// update works on x + xlo in FP32 and splits the result back, so steps smaller
// than half an ulp of x still accumulate instead of being rounded away.
template <typename T>
__device__ __forceinline__ float updated(const T *x, const T *xlo, int64_t k, float mu, float g,
                                         T *xo, T *xloo) {
    if (xlo == nullptr) {
        const float nv = fmaf(mu, g, ldv(x + k));
        stf(xo + k, nv);
        return rnd(nv, xo);
    }
    const float s = fmaf(mu, g, ldv(x + k) + ldv(xlo + k));
    const float hi = rnd(s, xo);
    stf(xo + k, hi);
    stf(xloo + k, s - hi);
    return hi;
}

// Work of column block c of the iteration, shared by `nblk` CTAs of 256 threads
// (this one is `blk`). Without the y-fastest copies: a strided pass over the
// slab. With them: 32 x 32 (y, x) tiles of each z plane, where the gradient is
// g + transpose(gT) and the new x is also written transposed into xT, both
// transposes staged through shared memory so every global access is coalesced.
template <typename T>
__device__ void update_body(const DeviceGeom &G, const SolveDev &S, T *__restrict__ x,
                            T *__restrict__ xlo, int c, int blk, int nblk) {
    const Work &W = *S.work;
    if (c >= W.n_cols) return;
    const int j = W.cols[c];
    if (S.owned && !S.owned[j]) return;   // another process owns block j
    const float mu = (float)*S.mu;
    if (S.gT == nullptr) {
        const int64_t b0 = (int64_t)G.plane_start[j] * G.plane_stride;
        const int64_t b1 = (int64_t)G.plane_start[j + 1] * G.plane_stride;
        for (int64_t k = b0 + (int64_t)blk * blockDim.x + threadIdx.x; k < b1;
             k += (int64_t)nblk * blockDim.x) {
            const float gv = S.g[k];
            updated(x, xlo, k, mu, gv, x, xlo);
            if (S.eud) S.eud[k] += gv;
        }
        return;
    }
    __shared__ float sg[32][33];
    __shared__ float sx[32][33];
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;   // 32 x 8 threads
    const int nx = G.nx, ny = G.ny;
    const int tx_n = (nx + 31) / 32, ty_n = (ny + 31) / 32;
    const int z0 = G.plane_start[j], nzj = G.plane_start[j + 1] - z0;
    const int ntiles = tx_n * ty_n * nzj;
    T *xT = reinterpret_cast<T *>(S.xT);
    for (int t = blk; t < ntiles; t += nblk) {
        const int z = z0 + t / (tx_n * ty_n), rem = t % (tx_n * ty_n);
        const int x0 = (rem % tx_n) * 32, y0 = (rem / tx_n) * 32;
        // tile bases: [z][x][y] for gT / xT, [z][y][x] for x, g, xlo, eud
        const int64_t plane = (int64_t)z * nx * ny;
        const int64_t bT = plane + (int64_t)x0 * ny + y0;   // + k * ny + lane
        const int64_t bX = plane + (int64_t)y0 * nx + x0;   // + k * nx + lane
        const bool full = x0 + 32 <= nx && y0 + 32 <= ny;
        // every global load of the tile first (the gT rows to transpose, this
        // thread's g and x values): one round of memory latency per tile
        float gt[4], gv[4], xs[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = row + 8 * q;
            const bool inT = full || (x0 + k < nx && y0 + lane < ny);   // gT rows: fixed x
            gt[q] = inT ? S.gT[bT + k * ny + lane] : 0.f;
            const bool inX = full || (y0 + k < ny && x0 + lane < nx);   // x rows: fixed y
            const int64_t idx = bX + k * nx + lane;
            gv[q] = inX ? S.g[idx] : 0.f;
            xs[q] = inX ? (xlo ? ldv(x + idx) + ldv(xlo + idx) : ldv(x + idx)) : 0.f;
        }
        __syncthreads();   // the previous tile's xT stores are done with sx
#pragma unroll
        for (int q = 0; q < 4; ++q) sg[row + 8 * q][lane] = gt[q];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = row + 8 * q;
            if (full || (y0 + k < ny && x0 + lane < nx)) {
                const int64_t idx = bX + k * nx + lane;
                const float g = gv[q] + sg[lane][k];
                const float s = fmaf(mu, g, xs[q]);
                const float hi = rnd(s, x);
                stf(x + idx, hi);
                if (xlo) stf(xlo + idx, s - hi);
                sx[k][lane] = hi;
                if (S.eud) S.eud[idx] += g;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = row; k < 32; k += 8) {           // xT rows: fixed x, consecutive y
            if (full || (x0 + k < nx && y0 + lane < ny)) stf(xT + bT + k * ny + lane, sx[lane][k]);
        }
    }
}

// The block update of this iteration and the draw of the next (the first
// `dc` CTAs of row 0, dispatched first, so that the draw runs beside the
// update instead of after it). With dc > 1 (residual-weighted pairs) the draw
// CTAs split the pair weights between them and the last one to finish (an
// atomic ticket) takes the draw: the FP64 sums are spread over dc SMs.
template <typename T>
__global__ void __launch_bounds__(256) update_sample_kernel(const DeviceGeom G, const SolveDev S,
                                                            T *__restrict__ x, T *__restrict__ xlo,
                                                            const SampleArgs An, int dc,
                                                            double *wscratch, unsigned *ticket) {
    if ((int)blockIdx.x < dc) {
        if (blockIdx.y != 0) return;
        if (dc == 1) {
            sample_body(An);
            return;
        }
        const int MN = G.M * G.N;
        const int per = (MN + dc - 1) / dc;
        const int k0 = min(MN, (int)blockIdx.x * per), k1 = min(MN, k0 + per);
        pair_weights(An, An.S, k0, k1, wscratch);
        __threadfence();
        __syncthreads();
        __shared__ unsigned s_last;
        if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == (unsigned)dc - 1;
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        sample_body(An, wscratch);
        if (threadIdx.x == 0) *ticket = 0u;
        return;
    }
    update_body<T>(G, S, x, xlo, blockIdx.y, blockIdx.x - dc, gridDim.x - dc);
}

// xT = transpose(x) over the whole volume (y fastest), through shared memory.
template <typename T>
__global__ void transpose_kernel(const DeviceGeom G, const T *__restrict__ x, T *__restrict__ xT) {
    __shared__ float sx[32][33];
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int tx_n = (G.nx + 31) / 32, ty_n = (G.ny + 31) / 32;
    const int ntiles = tx_n * ty_n * G.nz;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int z = t / (tx_n * ty_n), rem = t % (tx_n * ty_n);
        const int x0 = (rem % tx_n) * 32, y0 = (rem / tx_n) * 32;
        __syncthreads();
        for (int k = row; k < 32; k += 8) {
            const int yy = y0 + k, xx = x0 + lane;
            if (xx < G.nx && yy < G.ny) sx[k][lane] = ldv(x + ((int64_t)z * G.ny + yy) * G.nx + xx);
        }
        __syncthreads();
        for (int k = row; k < 32; k += 8) {
            const int xx = x0 + k, yy = y0 + lane;
            if (xx < G.nx && yy < G.ny) stf(xT + ((int64_t)z * G.nx + xx) * G.ny + yy, sx[lane][k]);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) update_kernel(const DeviceGeom G, const SolveDev S,
                                                     T *__restrict__ x, T *__restrict__ xlo) {
    update_body<T>(G, S, x, xlo, blockIdx.y, blockIdx.x, gridDim.x);
}

// Serving rounds. A request's draws alternate between two work lists: the
// round's passes use list 0; CTA 0 of the request's row of the update launch
// draws the next iteration into list 1 (its draw needs only the residual
// table, final once the round's FPs are done), so the draw runs beside the
// update as in bsgd_block_step; then the promote launch copies list 1 into
// list 0. The first draw of a request is made at its admission. No draw is
// made past the request's last iteration.
__global__ void __launch_bounds__(256) round_update_kernel(const ReqDesc *__restrict__ T,
                                                           const RoundCtl *__restrict__ C) {
    const int r = blockIdx.y;
    if (r >= C->n || !T[r].active || round_skips(T[r].period, C->round)) return;
    const ReqDesc &q = T[r];
    if (blockIdx.x == 0) {
        if (*q.A.iter < q.target) sample_body(q.A);
        return;
    }
    for (int c = 0; c < q.kN; ++c) {   // every drawn column block
        if (q.dtype == BSGD_F32)
            update_body<float>(q.G, q.S, (float *)q.x, nullptr, c, blockIdx.x - 1, gridDim.x - 1);
        else if (q.dtype == BSGD_BF16)
            update_body<__nv_bfloat16>(q.G, q.S, (__nv_bfloat16 *)q.x, (__nv_bfloat16 *)q.xlo, c,
                                       blockIdx.x - 1, gridDim.x - 1);
        else
            update_body<__half>(q.G, q.S, (__half *)q.x, (__half *)q.xlo, c, blockIdx.x - 1,
                                gridDim.x - 1);
    }
}

// List 1 (the next iteration's draw) into list 0, one CTA per request.
__global__ void __launch_bounds__(256) round_promote_kernel(const ReqDesc *__restrict__ T,
                                                            const RoundCtl *__restrict__ C) {
    const int r = blockIdx.x;
    if (r >= C->n || !T[r].active || round_skips(T[r].period, C->round)) return;
    const ReqDesc &q = T[r];
    const int *src = reinterpret_cast<const int *>(q.A.work);
    int *dst = reinterpret_cast<int *>(const_cast<Work *>(q.S.work));
    static_assert(sizeof(Work) % 4 == 0, "word copy");
    for (int k = threadIdx.x; k < (int)(sizeof(Work) / 4); k += blockDim.x) dst[k] = src[k];
    const int nc = kMaxPairs * q.G.max_views;
    int *cdst = const_cast<int *>(q.S.cells);
    for (int k = threadIdx.x; k < nc; k += blockDim.x) cdst[k] = q.A.cells[k];
}

// The round's last node: every kernel of the round has read its index.
__global__ void round_tick_kernel(RoundCtl *C) { C->round += 1ull; }

bsgd_status launch_round_update(const ReqDesc *table, RoundCtl *ctl, int max_slots,
                                cudaStream_t st) {
    round_update_kernel<<<dim3(152 * 2 + 1, max_slots), 256, 0, st>>>(table, ctl);
    round_promote_kernel<<<max_slots, 256, 0, st>>>(table, ctl);
    round_tick_kernel<<<1, 1, 0, st>>>(ctl);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

// S[block(a)][v] += r^2 over all rows (the FP64 residual table from scratch).
template <typename T>
__global__ void norm_table_kernel(const DeviceGeom G, const T *__restrict__ r, double *S) {
    const int64_t per_row = G.nu;
    const int64_t n_lines = (int64_t)G.n_views * G.nv;
    for (int64_t line = blockIdx.x; line < n_lines; line += gridDim.x) {
        const int a = (int)(line / G.nv), v = (int)(line % G.nv);
        double acc = 0.0;
        for (int64_t u = threadIdx.x; u < per_row; u += blockDim.x) {
            const float x = ldv(r + line * per_row + u);
            acc += (double)x * x;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0 && acc != 0.0)
            atomicAdd(S + (size_t)G.view_block[a] * G.nv + v, acc);
    }
}

template <typename TI, typename TO>
__global__ void convert_kernel(const TI *__restrict__ in, TO *__restrict__ out, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        stf(out + k, ldf(in + k));
}

// Per (view, cell) sums of an FP of block J's indicator (FP64), then the floor.
__global__ void cell_sum_kernel(const DeviceGeom G, const float *__restrict__ yj, int j,
                                int n_cells, double *cw) {
    const int64_t n = G.n_rows;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        const float val = yj[row];
        if (val == 0.f) continue;
        const int u = (int)(row % G.nu), v = (int)((row / G.nu) % G.nv);
        const int a = (int)(row / ((int64_t)G.nu * G.nv));
        int c = 0;
        if (n_cells == 2) c = u >= G.nu / 2;
        if (n_cells == 4) c = (v >= G.nv / 2) * 2 + (u >= G.nu / 2);
        atomicAdd(cw + ((size_t)j * G.n_views + a) * n_cells + c, (double)val);
    }
}

__global__ void cell_floor_kernel(const DeviceGeom G, int n_cells, double *cw) {
    const int64_t n = (int64_t)G.N * G.n_views;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        double *w = cw + k * n_cells;
        double tot = 0.0;
        for (int s = 0; s < n_cells; ++s) tot += w[s];
        for (int s = 0; s < n_cells; ++s) w[s] = fmax(w[s], kCellFloor * tot);
    }
}

// ---- power iteration helpers (FP64 vector state) --------------------------

__global__ void sumsq_kernel(const float *__restrict__ a, int64_t b0, int64_t b1, double *out) {
    double acc = 0.0;
    for (int64_t k = b0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < b1;
         k += (int64_t)gridDim.x * blockDim.x)
        acc += (double)a[k] * a[k];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(out, acc);
    }
}

// v = w / ||w|| (FP64) on [b0, b1); v32 = float(v); zero w.
__global__ void normalize_kernel(float *__restrict__ w, double *__restrict__ v64,
                                 float *__restrict__ v32, int64_t b0, int64_t b1,
                                 const double *nrm2, int init) {
    const double inv = init ? 1.0 / sqrt((double)(b1 - b0)) : 1.0 / sqrt(*nrm2);
    for (int64_t k = b0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < b1;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double v = init ? inv : (double)w[k] * inv;
        v64[k - b0] = v;
        v32[k] = (float)v;
        w[k] = 0.f;
    }
}

int grid_for(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace bsgd

using namespace bsgd;

// ---------------------------------------------------------------------------
// State

// ---------------------------------------------------------------------------
// Algorithm 3: automatic step length. The update kernel adds every applied
// direction g_J into eud; at the end of a window the two FP64 reductions below
// give <eud, eud_prev>, ||eud||^2, ||eud_prev||^2 and ||r||^2 = sum S, and one
// thread applies the test to mu in device memory.

constexpr int kAutoParts = 608;   // reduction blocks (152 SMs x 4)

struct AutoMuHist {
    double rho_m1, rho_m2;   // ||r|| at the previous two window ends
    double theta_m1;         // cosine at the previous window end
    int have_theta_m1;       // theta_m1 defined
    int e;                   // windows completed
};

__device__ inline double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(256) automu_dot_kernel(const double *__restrict__ a,
                                                         const double *__restrict__ b, int64_t n,
                                                         double *__restrict__ part) {
    __shared__ double sh[8];
    double d = 0.0, na = 0.0, nb = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double u = a[k], v = b[k];
        d = fma(u, v, d);
        na = fma(u, u, na);
        nb = fma(v, v, nb);
    }
    d = block_sum(d, sh);
    na = block_sum(na, sh);
    nb = block_sum(nb, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = d;
        part[3 * blockIdx.x + 1] = na;
        part[3 * blockIdx.x + 2] = nb;
    }
}

// ||r|| from the FP64 residual table (sum over row blocks and detector rows)
__device__ inline double table_norm(const double *S, int nS, double *sh) {
    double t = 0.0;
    for (int k = threadIdx.x; k < nS; k += blockDim.x) t += S[k];
    t = block_sum(t, sh);
    return sqrt(fmax(t, 0.0));
}

__global__ void __launch_bounds__(256) automu_init_kernel(const double *S, int nS, AutoMuHist *h) {
    __shared__ double sh[8];
    const double rho = table_norm(S, nS, sh);
    if (threadIdx.x == 0) {
        h->rho_m1 = rho;
        h->rho_m2 = 0.0;
        h->theta_m1 = 0.0;
        h->have_theta_m1 = 0;
        h->e = 0;
    }
}

__global__ void __launch_bounds__(256) automu_decide_kernel(const double *part, int nparts,
                                                            const double *S, int nS, AutoMuHist *h,
                                                            double *mu, double eps, double delta,
                                                            double t1, double t2) {
    __shared__ double sh[8];
    double d = 0.0, na = 0.0, nb = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
        d += part[3 * k];
        na += part[3 * k + 1];
        nb += part[3 * k + 2];
    }
    d = block_sum(d, sh);
    na = block_sum(na, sh);
    nb = block_sum(nb, sh);
    const double rho = table_norm(S, nS, sh);
    if (threadIdx.x != 0) return;
    const int e = ++h->e;
    const bool have_theta = e >= 2;   // the first window has no previous direction
    const double theta = !have_theta ? 0.0
                         : (na == 0.0 || nb == 0.0) ? 1.0 : d / (sqrt(na) * sqrt(nb));
    if (e >= 2) {
        const double r0 = h->rho_m2, r1 = h->rho_m1, r2 = rho;
        if (r2 < r1 && r1 < r0) {
            *mu *= 1.0 + eps;
        } else if (r2 > r1 && r1 > r0) {
            const bool c2 = theta < t2;
            const bool c1 = h->have_theta_m1 && fabs(theta - h->theta_m1) > t1;
            if (c1 || c2) *mu *= 1.0 - delta;
        }
    }
    h->rho_m2 = h->rho_m1;
    h->rho_m1 = rho;
    h->theta_m1 = theta;
    h->have_theta_m1 = have_theta;
}

struct bsgd_state {
    const bsgd_geometry *g = nullptr;
    bsgd_solve_params p{};
    int kM = 1, kN = 1, P = 1, epoch_len = 1;
    bsgd_dtype st = BSGD_F32;
    bool fused = true;
    int max_tiles = 0;
    int max_tiles_all = 0;      // tiles of the whole-volume band (bounds any union of bands)
    int n_cells = 1;
    int stride = 0;
    int64_t trace_cap = 0;
    int64_t iters = 0;          // iterations launched
    double mu = 0.0;
    // device memory
    void *y = nullptr, *z = nullptr, *rt = nullptr, *r = nullptr;
    void *xlo = nullptr;        // low-order image term (16-bit storage only)
    void *xT = nullptr;         // y-fastest copy of x (volumes only)
    float *gT = nullptr;        // y-fastest part of g (volumes only)
    float *grad = nullptr;
    double *S = nullptr, *cw = nullptr, *d_mu = nullptr;
    Work *work = nullptr;
    int *cells = nullptr, *wband = nullptr;
    int64_t *d_iter = nullptr;
    int *x0_flag = nullptr;     // warm start: 1 if the starting image is not zero
    double *wscratch = nullptr; // residual-pair weights of a split draw
    unsigned *ticket = nullptr; // the split draw's completion counter
    unsigned char *owned = nullptr;  // owner-computes sharding: owned column blocks (N)
    bool zero_start = false;    // the caller's image is known to be zero: no warm start
    int32_t *trace = nullptr, *replay = nullptr;
    int64_t replay_start = 0, replay_n = 0;
    unsigned long long *counts = nullptr, *updates = nullptr;
    unsigned long long *pair_upd = nullptr;   // M x N whole-view update counts
    // Algorithm 3
    int auto_win = 0;            // epochs per test (0: off)
    double *eud = nullptr, *eud_prev = nullptr, *am_part = nullptr;
    AutoMuHist *am = nullptr;
    TvWork tv;                   // BSGD-TV prox workspace (tv_lambda > 0)
    SolveDev dev{};
    // tracing: event pairs per stage (a pool reused after each read)
    bool profiling = false;
    bool split = false;          // run FP and BP as separate kernels (profiling aid)
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    int64_t launches[BSGD_N_STAGES] = {};
    double ms[BSGD_N_STAGES] = {};
};

static cudaEvent_t next_event(bsgd_state *s) {
    if (s->ev_used == s->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        s->ev_pool.push_back(e);
    }
    return s->ev_pool[s->ev_used++];
}

// Record the start of a stage; returns its begin event (or null when off).
static cudaEvent_t stage_begin(bsgd_state *s, cudaStream_t st) {
    if (!s->profiling) return nullptr;
    cudaEvent_t b = next_event(s);
    if (b) cudaEventRecord(b, st);
    return b;
}

static void stage_end(bsgd_state *s, int stage, cudaEvent_t b, int launches, cudaStream_t st) {
    if (!s->profiling || !b) return;
    cudaEvent_t e = next_event(s);
    if (!e) return;
    cudaEventRecord(e, st);
    s->marks.push_back({stage, {b, e}});
    s->launches[stage] += launches;
}

// Solver states and the one-call solver take their device memory from a
// stream-ordered pool per device that keeps up to kPoolKeep bytes of freed
// memory for reuse, so creating a state for every call costs no page mapping
// once the pool is warm (cudaMalloc / cudaFree of ~2 GB took ~4 ms per call).
constexpr uint64_t kPoolKeep = 32ull << 30;

static bsgd_status state_pool(cudaMemPool_t *out) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    BSGD_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(dev);
    if (it == pools.end()) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        BSGD_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = kPoolKeep;
        BSGD_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        it = pools.emplace(dev, pool).first;
    }
    *out = it->second;
    return BSGD_OK;
}

// Allocation from the pool, ordered on stream st.
static bsgd_status palloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    BSGD_TRY(state_pool(&pool));
    cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? BSGD_ERR_OOM : BSGD_ERR_CUDA,
                    std::string("pool allocation of ") + std::to_string(bytes) +
                        " bytes: " + cudaGetErrorString(e));
    }
    return BSGD_OK;
}

// Return pool memory; callers have synchronised the work that used it.
static void pfree(void *p) {
    if (p) cudaFreeAsync(p, 0);
}

namespace bsgd {
bsgd_status pool_alloc(void **p, size_t bytes, cudaStream_t st) { return palloc(p, bytes, st); }
bool pool_try_alloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    if (state_pool(&pool) != BSGD_OK) return false;
    if (cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, st) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}
void pool_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}
}  // namespace bsgd

static void free_state(bsgd_state *s) {
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    // counts and cw belong to the geometry's cache; replay is a plain allocation
    void *ptrs[] = {s->y, s->z, s->rt, s->r, s->xlo, s->xT, s->gT, s->grad, s->S, s->d_mu, s->work, s->cells,
                    s->wband, s->d_iter, s->x0_flag, s->owned, s->wscratch, s->ticket, s->trace,
                    s->updates, s->pair_upd, s->eud, s->eud_prev, s->am_part, s->am};
    for (void *p : ptrs) pfree(p);
    cudaFree(s->replay);
    tv_work_free(s->tv);
    delete s;
}

static bsgd_status dalloc(void **p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? BSGD_ERR_OOM : BSGD_ERR_CUDA,
                    std::string("cudaMalloc of ") + std::to_string(bytes) +
                        " bytes: " + cudaGetErrorString(e));
    }
    return BSGD_OK;
}

namespace bsgd {

bsgd_status convert(const void *in, bsgd_dtype it, void *out, bsgd_dtype ot, int64_t n,
                    cudaStream_t st) {
    if (it == ot) {
        BSGD_CUDA(cudaMemcpyAsync(out, in, n * dtype_size(it), cudaMemcpyDeviceToDevice, st));
        return BSGD_OK;
    }
    const int gb = grid_for(n);
#define CV(TI, TO) convert_kernel<TI, TO><<<gb, 256, 0, st>>>((const TI *)in, (TO *)out, n)
    if (it == BSGD_F32 && ot == BSGD_BF16) CV(float, __nv_bfloat16);
    else if (it == BSGD_F32 && ot == BSGD_F16) CV(float, __half);
    else if (it == BSGD_BF16 && ot == BSGD_F32) CV(__nv_bfloat16, float);
    else if (it == BSGD_BF16 && ot == BSGD_F16) CV(__nv_bfloat16, __half);
    else if (it == BSGD_F16 && ot == BSGD_F32) CV(__half, float);
    else CV(__half, __nv_bfloat16);
#undef CV
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status norm_table(const bsgd_geometry *g, const void *r, bsgd_dtype t, double *S,
                       cudaStream_t st) {
    BSGD_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * g->M * g->desc.nv, st));
    const int64_t lines = (int64_t)g->desc.n_views * g->desc.nv;
    const int gb = (int)std::min<int64_t>(lines, 152 * 32);
    if (t == BSGD_F32) norm_table_kernel<float><<<gb, 128, 0, st>>>(g->dg, (const float *)r, S);
    else if (t == BSGD_BF16) norm_table_kernel<__nv_bfloat16><<<gb, 128, 0, st>>>(g->dg, (const __nv_bfloat16 *)r, S);
    else norm_table_kernel<__half><<<gb, 128, 0, st>>>(g->dg, (const __half *)r, S);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

// lambda ~ ||A_rows^J||^2 by power iteration (see bsgd.h).
bsgd_status power_iteration(const bsgd_geometry *g, int j, int iters, const int *row_ids, int n_rb,
                            double *lambda, cudaStream_t st) {
    const int64_t b0 = (int64_t)g->plane_start[j] * g->dg.plane_stride;
    const int64_t b1 = (int64_t)g->plane_start[j + 1] * g->dg.plane_stride;
    const int64_t n = g->n_cols(), m = g->n_rows();
    float *v32 = nullptr, *w = nullptr, *y = nullptr, *vT = nullptr, *wT = nullptr;
    double *v64 = nullptr, *nrm = nullptr;
    bsgd_status s = BSGD_OK;
    auto cleanup = [&]() {
        for (void *p : {(void *)v32, (void *)w, (void *)y, (void *)v64, (void *)nrm, (void *)vT, (void *)wT})
            pool_free(p, st);
    };
    if ((s = palloc((void **)&v32, n * 4, st)) || (s = palloc((void **)&w, n * 4, st)) ||
        (s = palloc((void **)&y, m * 4, st)) || (s = palloc((void **)&v64, (b1 - b0) * 8, st)) ||
        (s = palloc((void **)&nrm, 8 * (iters + 2), st))) {
        cleanup();
        return s;
    }
    std::vector<int> all;
    if (!row_ids) {
        for (int i = 0; i < g->M; ++i) all.push_back(i);
        row_ids = all.data();
        n_rb = g->M;
    }
    // y-fastest copies of v and of the BP accumulator for the views whose rays
    // run along x (optional: without them the iteration is the same, slower)
    if (plain_wants_transpose(g, row_ids, n_rb) &&
        (!pool_try_alloc((void **)&vT, n * 4, st) || !pool_try_alloc((void **)&wT, n * 4, st))) {
        pool_free(vT, st);
        pool_free(wT, st);
        vT = wT = nullptr;
    }
    PlainLaunch L{row_ids, n_rb, j, j + 1, 0};
    // A^T A v over block j: FP of v, then BP into w (and wT, added back)
    auto ata = [&]() -> bsgd_status {
        BSGD_CUDA(cudaMemsetAsync(y, 0, m * 4, st));
        if (vT) BSGD_TRY(plain_transpose(g, v32, BSGD_F32, vT, j, j + 1, st));
        BSGD_TRY(launch_fp_plain(g, L, v32, BSGD_F32, y, BSGD_F32, 1, st, vT));
        if (wT) BSGD_CUDA(cudaMemsetAsync(wT + b0, 0, (b1 - b0) * 4, st));
        BSGD_TRY(launch_bp_plain(g, L, y, BSGD_F32, w, 1.0f, st, wT));
        if (wT) BSGD_TRY(plain_add_transposed(g, wT, w, j, j + 1, st));
        return BSGD_OK;
    };
    const int gb = grid_for(b1 - b0);
    auto run = [&]() -> bsgd_status {
        BSGD_CUDA(cudaMemsetAsync(v32, 0, n * 4, st));
        BSGD_CUDA(cudaMemsetAsync(w, 0, n * 4, st));
        BSGD_CUDA(cudaMemsetAsync(nrm, 0, 8 * (iters + 2), st));
        normalize_kernel<<<gb, 256, 0, st>>>(w, v64, v32, b0, b1, nrm, 1);
        for (int k = 0; k < iters; ++k) {
            BSGD_TRY(ata());
            sumsq_kernel<<<gb, 256, 0, st>>>(w, b0, b1, nrm + k);
            normalize_kernel<<<gb, 256, 0, st>>>(w, v64, v32, b0, b1, nrm + k, 0);
        }
        BSGD_CUDA(cudaMemsetAsync(y, 0, m * 4, st));
        if (vT) BSGD_TRY(plain_transpose(g, v32, BSGD_F32, vT, j, j + 1, st));
        BSGD_TRY(launch_fp_plain(g, L, v32, BSGD_F32, y, BSGD_F32, 1, st, vT));
        sumsq_kernel<<<grid_for(m), 256, 0, st>>>(y, 0, m, nrm + iters);
        BSGD_CUDA(cudaGetLastError());
        BSGD_CUDA(cudaMemcpyAsync(lambda, nrm + iters, 8, cudaMemcpyDeviceToHost, st));
        BSGD_CUDA(cudaStreamSynchronize(st));
        return BSGD_OK;
    };
    s = run();
    cleanup();
    return s;
}

}  // namespace bsgd

extern "C" bsgd_status bsgd_power_iteration(const bsgd_geometry *g, int col_block, int iters,
                                            const int32_t *row_blocks, int n_rb,
                                            double *lambda_out, void *stream) {
    if (!g || !lambda_out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (col_block < 0 || col_block >= g->N) return fail(BSGD_ERR_INVALID_ARG, "col_block out of range");
    if (iters < 0) return fail(BSGD_ERR_INVALID_ARG, "iters < 0");
    BSGD_TRY(check_device(g));
    if (row_blocks)
        for (int k = 0; k < n_rb; ++k)
            if (row_blocks[k] < 0 || row_blocks[k] >= g->M)
                return fail(BSGD_ERR_INVALID_ARG, "row block id out of range");
    return power_iteration(g, col_block, iters, (const int *)row_blocks, row_blocks ? n_rb : 0,
                           lambda_out, (cudaStream_t)stream);
}

static bsgd_status check_params(const bsgd_geometry *g, const bsgd_solve_params *p) {
    if (!(p->alpha > 0 && p->alpha <= 1) || !(p->gamma > 0 && p->gamma <= 1))
        return fail(BSGD_ERR_INVALID_ARG, "alpha and gamma must lie in (0, 1]");
    if (!dtype_ok(p->storage)) return fail(BSGD_ERR_INVALID_ARG, "bad storage dtype");
    if (p->step_rule < BSGD_STEP_STRIP || p->step_rule > BSGD_STEP_FIXED)
        return fail(BSGD_ERR_INVALID_ARG, "bad step rule");
    if (p->step_rule == BSGD_STEP_FIXED && !(p->mu > 0))
        return fail(BSGD_ERR_INVALID_ARG, "fixed step needs mu > 0");
    if (p->step_rule != BSGD_STEP_FIXED && (!(p->rho > 0) || p->power_iters < 1))
        return fail(BSGD_ERR_INVALID_ARG, "STRIP / BLOCK steps need rho > 0 and power_iters >= 1");
    if (p->pair_sampling != BSGD_PAIRS_UNIFORM && p->pair_sampling != BSGD_PAIRS_RESIDUAL)
        return fail(BSGD_ERR_INVALID_ARG, "bad pair sampling");
    if (p->cells < BSGD_CELLS_NONE || p->cells > BSGD_CELLS_UNIFORM)
        return fail(BSGD_ERR_INVALID_ARG, "bad cell sampling");
    if (p->cells != BSGD_CELLS_NONE && p->n_cells != (g->desc.nv > 1 ? 4 : 2))
        return fail(BSGD_ERR_INVALID_ARG, "n_cells must be 4 (3D) or 2 (2D)");
    if (g->M > kMaxSampleBlocks || g->N > kMaxSampleBlocks || g->M > 64)
        return fail(BSGD_ERR_INVALID_ARG, "the solver supports M <= 64 and N <= 1024");
    if (p->pair_sampling == BSGD_PAIRS_RESIDUAL && g->M * g->N > kMaxResidualPairs)
        return fail(BSGD_ERR_INVALID_ARG, "residual sampling supports M * N <= 1024");
    if (p->tv_lambda < 0 || (p->tv_lambda > 0 && p->tv_iters < 1))
        return fail(BSGD_ERR_INVALID_ARG, "tv_lambda >= 0 and tv_iters >= 1");
    if (p->tv_lambda > 0 && g->desc.nz > 65535)
        return fail(BSGD_ERR_INVALID_ARG, "the TV prox supports nz <= 65535");
    if (p->auto_mu) {
        if (!(p->auto_eps > 0) || !(p->auto_delta > 0 && p->auto_delta < 1) || !(p->auto_t1 > 0) ||
            p->auto_window < 0 || !std::isfinite(p->auto_t2))
            return fail(BSGD_ERR_INVALID_ARG,
                        "automatic step: auto_eps > 0, 0 < auto_delta < 1, auto_t1 > 0, auto_window >= 0");
        if (p->tv_lambda > 0)
            return fail(BSGD_ERR_INVALID_ARG, "the automatic step is not combined with the TV prox");
    }
    return BSGD_OK;
}


// Update counts per (J, view, cell) and, for Algorithm 2, the geometric cell
// weights w(a, c, J) = 1^T A_(a,c)^J 1 (an FP of J's indicator summed per
// cell): computed once per geometry and cell count, then shared by every
// state of the geometry (read-only).
static bsgd_status geometry_tables(const bsgd_geometry *g, int n_cells, bool weights,
                                   cudaStream_t st, unsigned long long **counts, double **cw) {
    std::lock_guard<std::mutex> lock(g->cache_mu);
    const int N = g->N, M = g->M, V = g->desc.n_views;
    const int64_t R = g->n_rows(), C = g->n_cols();
    if (!g->d_counts[n_cells]) {
        unsigned long long *c = nullptr;
        BSGD_TRY(dalloc((void **)&c, 8 * (size_t)N * V * n_cells));
        bsgd_status e = BSGD_OK;
        if (cudaMemsetAsync(c, 0, 8 * (size_t)N * V * n_cells, st) != cudaSuccess)
            e = fail(BSGD_ERR_CUDA, "cudaMemsetAsync failed");
        for (int j = 0; j < N && !e; ++j)
            e = launch_count_cells(g, j, n_cells, c + (size_t)j * V * n_cells, st);
        if (!e && cudaStreamSynchronize(st) != cudaSuccess) e = fail(BSGD_ERR_CUDA, "count pass failed");
        if (e) {
            cudaStreamSynchronize(st);
            cudaFree(c);
            return e;
        }
        g->d_counts[n_cells] = c;
    }
    *counts = g->d_counts[n_cells];
    *cw = nullptr;
    if (!weights) return BSGD_OK;
    if (!g->d_cw[n_cells]) {
        double *w = nullptr;
        float *ind = nullptr, *yj = nullptr;
        BSGD_TRY(dalloc((void **)&w, 8 * (size_t)N * V * n_cells));
        bsgd_status e = dalloc((void **)&ind, C * 4);
        if (!e) e = dalloc((void **)&yj, R * 4);
        if (!e && cudaMemsetAsync(w, 0, 8 * (size_t)N * V * n_cells, st) != cudaSuccess)
            e = fail(BSGD_ERR_CUDA, "cudaMemsetAsync failed");
        std::vector<int> all(M);
        for (int i = 0; i < M; ++i) all[i] = i;
        std::vector<float> ones;
        for (int j = 0; j < N && !e; ++j) {
            cudaMemsetAsync(ind, 0, C * 4, st);
            const int64_t b0 = (int64_t)g->plane_start[j] * g->dg.plane_stride;
            ones.assign(g->block_cols(j), 1.0f);
            cudaMemcpyAsync(ind + b0, ones.data(), ones.size() * 4, cudaMemcpyHostToDevice, st);
            cudaStreamSynchronize(st);
            cudaMemsetAsync(yj, 0, R * 4, st);
            PlainLaunch L{all.data(), M, j, j + 1, 0};
            e = launch_fp_plain(g, L, ind, BSGD_F32, yj, BSGD_F32, 1, st);
            if (!e) cell_sum_kernel<<<grid_for(R), 256, 0, st>>>(g->dg, yj, j, n_cells, w);
        }
        if (!e) cell_floor_kernel<<<grid_for((int64_t)N * V), 256, 0, st>>>(g->dg, n_cells, w);
        if (cudaStreamSynchronize(st) != cudaSuccess && !e) e = fail(BSGD_ERR_CUDA, "cell weights failed");
        if (!e && cudaGetLastError() != cudaSuccess) e = fail(BSGD_ERR_CUDA, "cell weights failed");
        cudaFree(ind);
        cudaFree(yj);
        if (e) {
            cudaFree(w);
            return e;
        }
        g->d_cw[n_cells] = w;
    }
    *cw = g->d_cw[n_cells];
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_state_create(const bsgd_geometry *g, const bsgd_solve_params *p,
                                         const void *y, bsgd_dtype yt, void *stream,
                                         bsgd_state **out) {
    if (!g || !p || !y || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (!dtype_ok(yt)) return fail(BSGD_ERR_INVALID_ARG, "bad y dtype");
    BSGD_TRY(check_params(g, p));
    BSGD_TRY(check_device(g));
    cudaStream_t st = (cudaStream_t)stream;
    bsgd_state *s = new (std::nothrow) bsgd_state();
    if (!s) return fail(BSGD_ERR_OOM, "host allocation failed");
    s->g = g;
    s->p = *p;
    s->kM = std::max(1, (int)std::lround(p->alpha * g->M));
    s->kN = std::max(1, (int)std::lround(p->gamma * g->N));
    s->P = s->kM * s->kN;
    s->epoch_len = std::max(1, (int)std::lround(1.0 / (p->alpha * p->gamma)));
    s->st = (bsgd_dtype)p->storage;
    s->fused = s->kN == 1;
    s->n_cells = p->cells == BSGD_CELLS_NONE ? 1 : p->n_cells;
    if (s->P > kMaxPairs) {
        free_state(s);
        return fail(BSGD_ERR_INVALID_ARG, "more than 64 pairs per iteration");
    }
    if (p->pair_sampling == BSGD_PAIRS_RESIDUAL && s->P != 1) {
        free_state(s);
        return fail(BSGD_ERR_INVALID_ARG, "residual pair sampling draws one pair per iteration");
    }
    s->stride = 1 + 2 * s->P + s->P * g->max_views;
    s->trace_cap = 65536;
    const int64_t R = g->n_rows(), C = g->n_cols();
    const size_t es = dtype_size(s->st);
    const int N = g->N, M = g->M, V = g->desc.n_views;
    bsgd_status e = BSGD_OK;
    const int64_t Z = g->zlen;   // compact band storage of z^j and r~^j
    if ((e = palloc(&s->y, R * es, st)) || (e = palloc(&s->z, (size_t)Z * es, st)) ||
        (e = palloc(&s->rt, (size_t)Z * es, st)) || (e = palloc(&s->r, R * es, st)) ||
        (e = palloc((void **)&s->grad, C * 4, st)) || (e = palloc((void **)&s->S, 8 * (size_t)M * g->desc.nv, st)) ||
        (e = palloc((void **)&s->d_mu, 8, st)) || (e = palloc((void **)&s->work, 2 * sizeof(Work), st)) ||
        (e = palloc((void **)&s->cells, 2 * 4 * (size_t)kMaxPairs * g->max_views, st)) ||
        (e = palloc((void **)&s->wband, 4 * g->wband.size(), st)) ||
        (e = palloc((void **)&s->d_iter, 8, st)) || (e = palloc((void **)&s->x0_flag, 8, st)) ||
        (e = palloc((void **)&s->wscratch, 8 * (size_t)kMaxResidualPairs, st)) ||
        (e = palloc((void **)&s->ticket, 8, st)) ||
        (e = palloc((void **)&s->trace, 4 * (size_t)s->trace_cap * s->stride, st)) ||
        (e = palloc((void **)&s->updates, 8, st)) ||
        (e = palloc((void **)&s->pair_upd, 8 * (size_t)M * N, st)) ||
        (s->st != BSGD_F32 && !p->image_plain && (e = palloc(&s->xlo, C * es, st))) ||
        (g->desc.nz > 1 && (e = palloc(&s->xT, C * es, st))) ||
        (g->desc.nz > 1 && (e = palloc((void **)&s->gT, C * 4, st))) ||
        (p->tv_lambda > 0 && (e = tv_work_alloc(g, s->tv))) ||
        (p->auto_mu && ((e = palloc((void **)&s->eud, 8 * (size_t)C, st)) ||
                        (e = palloc((void **)&s->eud_prev, 8 * (size_t)C, st)) ||
                        (e = palloc((void **)&s->am_part, 8 * 3 * (size_t)kAutoParts, st)) ||
                        (e = palloc((void **)&s->am, sizeof(AutoMuHist), st))))) {
        cudaStreamSynchronize(st);
        free_state(s);
        return e;
    }
    auto init = [&]() -> bsgd_status {
        BSGD_TRY(convert(y, yt, s->y, s->st, R, st));
        BSGD_CUDA(cudaMemcpyAsync(s->r, s->y, R * es, cudaMemcpyDeviceToDevice, st));
        BSGD_CUDA(cudaMemsetAsync(s->z, 0, (size_t)Z * es, st));
        BSGD_CUDA(cudaMemsetAsync(s->rt, 0, (size_t)Z * es, st));
        BSGD_CUDA(cudaMemsetAsync(s->grad, 0, C * 4, st));
        if (s->xlo) BSGD_CUDA(cudaMemsetAsync(s->xlo, 0, C * es, st));
        if (s->xT) BSGD_CUDA(cudaMemsetAsync(s->xT, 0, C * es, st));
        if (s->gT) BSGD_CUDA(cudaMemsetAsync(s->gT, 0, C * 4, st));
        BSGD_CUDA(cudaMemsetAsync(s->d_iter, 0, 8, st));
        BSGD_CUDA(cudaMemsetAsync(s->ticket, 0, 8, st));
        BSGD_CUDA(cudaMemsetAsync(s->updates, 0, 8, st));
        BSGD_CUDA(cudaMemsetAsync(s->work, 0, 2 * sizeof(Work), st));
        BSGD_CUDA(cudaMemsetAsync(s->cells, 0xff, 2 * 4 * (size_t)kMaxPairs * g->max_views, st));
        BSGD_CUDA(cudaMemcpyAsync(s->wband, g->wband.data(), 4 * g->wband.size(),
                                  cudaMemcpyHostToDevice, st));
        BSGD_TRY(norm_table(g, s->r, s->st, s->S, st));
        BSGD_TRY(geometry_tables(g, s->n_cells, p->cells == BSGD_CELLS_GEOMETRIC, st, &s->counts, &s->cw));
        pair_updates_kernel<<<(M * N + 127) / 128, 128, 0, st>>>(g->dg, s->counts, s->n_cells, s->pair_upd);
        BSGD_CUDA(cudaGetLastError());
        // step size
        if (p->step_rule == BSGD_STEP_FIXED) {
            s->mu = p->mu;
        } else {
            const std::pair<int, int> key(p->step_rule, p->power_iters);
            double lmax = 0.0;
            bool cached = false;
            {
                std::lock_guard<std::mutex> lock(g->cache_mu);
                auto it = g->lambda_cache.find(key);
                if (it != g->lambda_cache.end()) {
                    lmax = it->second;
                    cached = true;
                }
            }
            for (int j = 0; j < N && !cached; ++j) {
                if (p->step_rule == BSGD_STEP_STRIP) {
                    double lam = 0.0;
                    BSGD_TRY(power_iteration(g, j, p->power_iters, nullptr, 0, &lam, st));
                    lmax = std::max(lmax, lam);
                } else {
                    for (int i = 0; i < M; ++i) {
                        double lam = 0.0;
                        BSGD_TRY(power_iteration(g, j, p->power_iters, &i, 1, &lam, st));
                        lmax = std::max(lmax, lam);
                    }
                }
            }
            if (!(lmax > 0)) return fail(BSGD_ERR_INVALID_ARG, "A^J is zero for every block");
            {
                std::lock_guard<std::mutex> lock(g->cache_mu);
                g->lambda_cache.emplace(key, lmax);
            }
            s->mu = p->rho / lmax;
        }
        BSGD_CUDA(cudaMemcpyAsync(s->d_mu, &s->mu, 8, cudaMemcpyHostToDevice, st));
        if (p->auto_mu) {
            s->auto_win = p->auto_window > 0 ? p->auto_window : M;
            BSGD_CUDA(cudaMemsetAsync(s->eud, 0, 8 * (size_t)C, st));
            BSGD_CUDA(cudaMemsetAsync(s->eud_prev, 0, 8 * (size_t)C, st));
            automu_init_kernel<<<1, 256, 0, st>>>(s->S, M * g->desc.nv, s->am);
            BSGD_CUDA(cudaGetLastError());
        }
        BSGD_CUDA(cudaStreamSynchronize(st));
        return BSGD_OK;
    };
    if ((e = init())) {
        cudaStreamSynchronize(st);
        free_state(s);
        return e;
    }
    std::vector<int> all(V);
    for (int a = 0; a < V; ++a) all[a] = a;
    for (int j = 0; j < N; ++j)
        s->max_tiles = std::max(s->max_tiles, tiles_for(g, all, j, j + 1, tile_u(g), tile_v(g)));
    s->max_tiles_all = tiles_for(g, all, 0, N, tile_u(g), tile_v(g));
    if ((int64_t)s->max_tiles_all * g->max_views > 0x7fffffff) {
        free_state(s);
        return fail(BSGD_ERR_INVALID_ARG, "detector tiles x views per block exceed one launch grid");
    }
    SolveDev &d = s->dev;
    d.y = s->y;
    d.z = s->z;
    d.rt = s->rt;
    d.r = s->r;
    d.g = s->grad;
    d.S = s->S;
    d.work = s->work;
    d.cells = s->cells;
    d.n_cells = s->n_cells;
    d.mu = s->d_mu;
    d.xT = s->xT;
    d.gT = s->gT;
    d.eud = s->eud;
    *out = s;
    return BSGD_OK;
}

namespace bsgd {
// Release a state whose work on stream st is the last that used it (serving):
// its pool memory is freed in stream order on st, without a device-wide
// synchronisation. States with TV workspace or a replay buffer synchronise st.
void state_release(bsgd_state *s, cudaStream_t st) {
    if (!s) return;
    if (s->tv.b || s->replay) {
        cudaStreamSynchronize(st);
        free_state(s);
        return;
    }
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    void *ptrs[] = {s->y, s->z, s->rt, s->r, s->xlo, s->xT, s->gT, s->grad, s->S, s->d_mu, s->work, s->cells,
                    s->wband, s->d_iter, s->x0_flag, s->owned, s->wscratch, s->ticket, s->trace,
                    s->updates, s->pair_upd, s->eud, s->eud_prev, s->am_part, s->am};
    for (void *p : ptrs) pool_free(p, st);
    delete s;
}
}  // namespace bsgd

extern "C" bsgd_status bsgd_state_destroy(bsgd_state *s) {
    if (!s) return fail(BSGD_ERR_INVALID_ARG, "state is NULL");
    cudaDeviceSynchronize();
    free_state(s);
    return BSGD_OK;
}

// The work list and the chosen cells are double-buffered by iteration parity,
// so the draw of iteration k + 1 can run while iteration k's update reads its
// own list.
static Work *work_buf(const bsgd_state *s, int64_t k) { return s->work + (k & 1); }
static int *cells_buf(const bsgd_state *s, int64_t k) {
    return s->cells + (k & 1) * (size_t)kMaxPairs * s->g->max_views;
}

static void fill_sample_args(const bsgd_state *s, SampleArgs &A, int64_t k) {
    const bsgd_geometry *g = s->g;
    A = SampleArgs{};
    A.it = k;
    A.G = g->dg;
    A.work = work_buf(s, k);
    A.cells = cells_buf(s, k);
    A.iter = s->d_iter;
    A.seed = s->p.seed;
    A.pairs_mode = s->p.pair_sampling;
    A.cells_mode = s->p.cells;
    A.n_cells = s->n_cells;
    A.kM = s->kM;
    A.kN = s->kN;
    A.S = s->S;
    A.wband = s->wband;
    A.cw = s->cw;
    A.replay = s->replay;
    A.replay_start = s->replay_start;
    A.replay_n = s->replay_n;
    A.trace = s->trace;
    A.trace_cap = s->trace_cap;
    A.stride = s->stride;
    A.counts = s->counts;
    A.pair_upd = s->pair_upd;
    A.updates = s->updates;
}

namespace bsgd {

// A served request's first draw (iteration 0, into list 0), on stream st.
bsgd_status state_first_draw(bsgd_state *s, cudaStream_t st) {
    SampleArgs A;
    fill_sample_args(s, A, 0);
    sample_kernel<<<1, kSampleThreads, 0, st>>>(A);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

bsgd_status state_descriptor(const bsgd_state *s, void *x, ReqDesc *out) {
    if (!s || !x || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!s->fused && (s->kN > kMaxFusedCols || s->p.pair_sampling != BSGD_PAIRS_UNIFORM))
        return fail(BSGD_ERR_INVALID_ARG, "serving takes at most 4 column blocks per iteration");
    if (s->p.tv_lambda > 0) return fail(BSGD_ERR_INVALID_ARG, "serving runs no TV prox");
    const bsgd_geometry *g = s->g;
    ReqDesc d{};
    d.G = g->dg;
    d.S = s->dev;
    d.S.work = work_buf(s, 0);   // served rounds solve and update with list 0
    d.S.cells = cells_buf(s, 0);
    fill_sample_args(s, d.A, 1);  // the next iteration's draw goes to list 1
    d.A.it = -1;                 // served rounds count iterations on the device
    d.x = x;
    d.xlo = s->xlo;
    d.dtype = s->st;
    // one block per iteration: items are (tile of the pair's band, view, pair);
    // several: (tile of the whole-volume band, view, drawn row block), as in
    // the multi-block fused pass
    d.kN = s->fused ? 1 : s->kN;
    const int tiles = s->fused ? s->max_tiles : s->max_tiles_all;
    d.max_tiles = std::max(1, tiles);
    d.active = s->max_tiles > 0 ? 1 : 0;
    d.period = 1;
    d.work_count = s->max_tiles > 0 ? (int64_t)tiles * g->max_views * (s->fused ? s->P : s->kM) : 0;
    int64_t maxJ = 0;
    for (int j = 0; j < g->N; ++j) maxJ = std::max(maxJ, g->block_cols(j));
    d.max_block_cols = maxJ;
    *out = d;
    return BSGD_OK;
}

size_t state_bytes(const bsgd_geometry_desc &d, int M, int N, const bsgd_solve_params &p,
                   size_t *transient) {
    const size_t R = (size_t)d.n_views * d.nu * d.nv, C = (size_t)d.nx * d.ny * d.nz;
    const size_t es = dtype_size((bsgd_dtype)p.storage);
    const int kM = std::max(1, (int)std::lround(p.alpha * M));
    const int kN = std::max(1, (int)std::lround(p.gamma * N));
    const int P = kM * kN;
    int maxV = (d.n_views + M - 1) / M;
    if (d.view_block) {
        std::vector<int> cnt(M, 0);
        for (int a = 0; a < d.n_views; ++a)
            if (d.view_block[a] >= 0 && d.view_block[a] < M) cnt[d.view_block[a]]++;
        maxV = *std::max_element(cnt.begin(), cnt.end());
    }
    const size_t cells = p.cells == BSGD_CELLS_NONE ? 1 : (size_t)std::max(1, p.n_cells);
    const size_t stride = 1 + 2 * (size_t)P + (size_t)P * maxV;
    // z^j and r~^j hold the rows of each block's band only (host tables)
    size_t Z = (size_t)N * R;
    {
        bsgd_geometry tmp;
        if (build_host_tables(&d, M, N, &tmp) == BSGD_OK) Z = (size_t)tmp.zlen;
    }
    size_t b = 0;
    b += R * es * 2 + Z * es * 2;                      // y, r, z^j, r~^j
    b += C * 4;                                        // g
    if (es != 4 && !p.image_plain) b += C * es;        // low-order image term
    if (d.nz > 1) b += C * (es + 4);                   // y-fastest copies of x and g
    b += 8 * (size_t)M * d.nv;                         // residual table
    b += 4 * (size_t)kMaxPairs * maxV + 8 * (size_t)M * N + sizeof(Work) + 64;
    b += 4 * (size_t)65536 * stride;                   // trace
    b += 8 * (size_t)N * d.n_views * cells * (p.cells == BSGD_CELLS_GEOMETRIC ? 2 : 1);
    // geometry tables
    b += 64 * (size_t)d.n_views + 16 * (size_t)d.n_views * (N + 1) + 4 * ((size_t)M * maxV + M + N + 1 + d.n_views);
    size_t t = 0;
    if (p.step_rule != BSGD_STEP_FIXED) t = std::max(t, C * 8 + R * 4 + C * 8 / N + 64);
    if (p.cells == BSGD_CELLS_GEOMETRIC) t = std::max(t, C * 4 + R * 4);
    t = std::max(t, 8 * (size_t)d.n_views);
    if (transient) *transient = t;
    return b;
}

}  // namespace bsgd

// xT = transpose(x): the caller's image is the one to trust at the start of
// every call (and after the TV prox rewrites it).
static bsgd_status sync_xT(bsgd_state *s, void *x, cudaStream_t st) {
    if (!s->xT) return BSGD_OK;
    const bsgd_geometry *g = s->g;
    const int tiles = ((g->desc.nx + 31) / 32) * ((g->desc.ny + 31) / 32) * g->desc.nz;
    const int gb = std::max(1, std::min(tiles, 152 * 8));
    if (s->st == BSGD_F32) transpose_kernel<float><<<gb, 256, 0, st>>>(g->dg, (const float *)x, (float *)s->xT);
    else if (s->st == BSGD_BF16) transpose_kernel<__nv_bfloat16><<<gb, 256, 0, st>>>(g->dg, (const __nv_bfloat16 *)x, (__nv_bfloat16 *)s->xT);
    else transpose_kernel<__half><<<gb, 256, 0, st>>>(g->dg, (const __half *)x, (__half *)s->xT);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

// The block update x_J += mu g_J of iteration s->iters (its work list); with
// draw_next, one extra CTA draws the next iteration's blocks.
static bsgd_status launch_update(bsgd_state *s, void *x, cudaStream_t st, bool draw_next) {
    const bsgd_geometry *g = s->g;
    const int64_t k = s->iters;
    int64_t maxJ = 0;
    for (int j = 0; j < g->N; ++j) maxJ = std::max(maxJ, g->block_cols(j));
    // with the y-fastest copies: one CTA per 32 x 32 tile of the slab
    const int64_t nt = s->gT ? ((g->desc.nx + 31) / 32) * (int64_t)((g->desc.ny + 31) / 32) *
                                   ((maxJ + (int64_t)g->desc.nx * g->desc.ny - 1) / ((int64_t)g->desc.nx * g->desc.ny))
                             : (maxJ + 1023) / 1024;
    // a grid of 4 CTAs per SM walks the tiles (the update is short: a second,
    // partial wave of one CTA per tile cost more than the loop)
    dim3 ug((unsigned)std::max<int64_t>(1, std::min<int64_t>(nt, 152 * 4)), s->kN);
    if (draw_next) {
        // the draw of iteration k + 1 needs only the residual table, final
        // once this iteration's FPs are done: one extra CTA of the update
        SampleArgs An;
        fill_sample_args(s, An, k + 1);
        // residual-weighted pairs (not replayed): the weights split over 8 CTAs
        const bool replay_next = s->replay && k + 1 >= s->replay_start && k + 1 < s->replay_start + s->replay_n;
        const int dc = (s->p.pair_sampling == BSGD_PAIRS_RESIDUAL && !replay_next &&
                        g->M * g->N >= 16) ? 8 : 1;
        dim3 ugs(ug.x + dc, ug.y);
        if (s->st == BSGD_F32)
            update_sample_kernel<float><<<ugs, 256, 0, st>>>(g->dg, s->dev, (float *)x, nullptr, An, dc,
                                                             s->wscratch, s->ticket);
        else if (s->st == BSGD_BF16)
            update_sample_kernel<__nv_bfloat16><<<ugs, 256, 0, st>>>(g->dg, s->dev, (__nv_bfloat16 *)x,
                                                                     (__nv_bfloat16 *)s->xlo, An, dc,
                                                                     s->wscratch, s->ticket);
        else
            update_sample_kernel<__half><<<ugs, 256, 0, st>>>(g->dg, s->dev, (__half *)x, (__half *)s->xlo,
                                                              An, dc, s->wscratch, s->ticket);
    } else {
        if (s->st == BSGD_F32) update_kernel<float><<<ug, 256, 0, st>>>(g->dg, s->dev, (float *)x, nullptr);
        else if (s->st == BSGD_BF16) update_kernel<__nv_bfloat16><<<ug, 256, 0, st>>>(g->dg, s->dev, (__nv_bfloat16 *)x, (__nv_bfloat16 *)s->xlo);
        else update_kernel<__half><<<ug, 256, 0, st>>>(g->dg, s->dev, (__half *)x, (__half *)s->xlo);
    }
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

// One iteration. `drawn`: its blocks were drawn by the previous iteration's
// update launch; `draw_next`: this iteration's update launch also draws the
// next iteration's blocks.
static bsgd_status one_iteration(bsgd_state *s, void *x, cudaStream_t st, bool drawn,
                                 bool draw_next) {
    const bsgd_geometry *g = s->g;
    const int64_t k = s->iters;
    s->dev.work = work_buf(s, k);
    s->dev.cells = cells_buf(s, k);
    cudaEvent_t b = nullptr;
    if (!drawn) {
        SampleArgs A;
        fill_sample_args(s, A, k);
        b = stage_begin(s, st);
        sample_kernel<<<1, kSampleThreads, 0, st>>>(A);
        BSGD_CUDA(cudaGetLastError());
        stage_end(s, BSGD_STAGE_SAMPLE, b, 1, st);
    }
    // several column blocks fuse too when every drawn row block is paired with
    // every drawn column block (uniform draws, not a replayed trace)
    const bool replaying = s->replay && k >= s->replay_start && k < s->replay_start + s->replay_n;
    const bool fuse_multi = !s->fused && s->kN <= kMaxFusedCols &&
                            s->p.pair_sampling == BSGD_PAIRS_UNIFORM && !replaying;
    if (s->max_tiles > 0 && s->fused && !s->split) {
        // one column block per iteration: FP, residual and BP in one pass
        b = stage_begin(s, st);
        BSGD_TRY(launch_fpbp_solve(g, s->dev, x, s->st, s->P, s->max_tiles, st));
        stage_end(s, BSGD_STAGE_FPBP, b, 1, st);
    } else if (s->max_tiles > 0 && fuse_multi && !s->split) {
        b = stage_begin(s, st);
        BSGD_TRY(launch_fpbpm_solve(g, s->dev, x, s->st, s->kM, s->max_tiles_all, s->kN, st));
        stage_end(s, BSGD_STAGE_FPBP, b, 1, st);
    } else if (s->max_tiles > 0) {
        b = stage_begin(s, st);
        BSGD_TRY(launch_fp_solve(g, s->dev, x, s->st, s->P, s->max_tiles, s->fused, st));
        stage_end(s, BSGD_STAGE_FP, b, 1, st);
        if (!s->fused) {
            b = stage_begin(s, st);
            dim3 grid((g->desc.nv + kResRows - 1) / kResRows, g->max_views, s->kM);
            if (s->st == BSGD_F32) residual_kernel<float><<<grid, 256, 0, st>>>(g->dg, s->dev);
            else if (s->st == BSGD_BF16) residual_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(g->dg, s->dev);
            else residual_kernel<__half><<<grid, 256, 0, st>>>(g->dg, s->dev);
            BSGD_CUDA(cudaGetLastError());
            stage_end(s, BSGD_STAGE_RESIDUAL, b, 1, st);
        }
        b = stage_begin(s, st);
        BSGD_TRY(launch_bp_solve(g, s->dev, s->st, s->P, s->max_tiles, st));
        stage_end(s, BSGD_STAGE_BP, b, 1, st);
    }
    b = stage_begin(s, st);
    BSGD_TRY(launch_update(s, x, st, draw_next));
    stage_end(s, BSGD_STAGE_UPDATE, b, 1, st);
    s->iters += 1;
    if (s->auto_win > 0 && s->iters % ((int64_t)s->epoch_len * s->auto_win) == 0) {
        // end of an Algorithm 3 window: test, then start the next direction
        const int64_t C = g->n_cols();
        automu_dot_kernel<<<kAutoParts, 256, 0, st>>>(s->eud, s->eud_prev, C, s->am_part);
        automu_decide_kernel<<<1, 256, 0, st>>>(s->am_part, kAutoParts, s->S, g->M * g->desc.nv,
                                                s->am, s->d_mu, s->p.auto_eps, s->p.auto_delta,
                                                s->p.auto_t1, s->p.auto_t2);
        BSGD_CUDA(cudaGetLastError());
        std::swap(s->eud, s->eud_prev);
        s->dev.eud = s->eud;
        BSGD_CUDA(cudaMemsetAsync(s->eud, 0, 8 * (size_t)C, st));
    }
    if (s->p.tv_lambda > 0 && s->iters % s->epoch_len == 0) {
        b = stage_begin(s, st);
        BSGD_TRY(tv_prox_run(g, x, s->st, s->mu * s->p.tv_lambda, s->p.tv_iters, st, s->xlo, s->tv));
        BSGD_TRY(sync_xT(s, x, st));
        stage_end(s, BSGD_STAGE_TV, b, 2 * s->p.tv_iters + 3, st);
    }
    return BSGD_OK;
}

// The first iteration of a state starts from the caller's image x0 (Algorithm 1
// starts from x0 = 0, z = 0, r = y): z^j = A^j x0_J for every block, r = y -
// sum_j z^j, then the residual table (and Algorithm 3's first residual norm)
// from that r; r~^j and g stay 0. All of it is skipped on the device when x0
// is zero.
static bsgd_status warm_start(bsgd_state *s, void *x, cudaStream_t st) {
    const bsgd_geometry *g = s->g;
    BSGD_TRY(launch_warm_start(g, s->dev, x, s->st, s->x0_flag, st));
    BSGD_TRY(norm_table(g, s->r, s->st, s->S, st));
    if (s->am) {
        automu_init_kernel<<<1, 256, 0, st>>>(s->S, g->M * g->desc.nv, s->am);
        BSGD_CUDA(cudaGetLastError());
    }
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_block_step(bsgd_state *s, void *x, int n_iters, void *stream) {
    if (!s || !x) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (n_iters < 0) return fail(BSGD_ERR_INVALID_ARG, "n_iters < 0");
    BSGD_TRY(check_device(s->g));
    cudaStream_t st = (cudaStream_t)stream;
    if (s->owned) return fail(BSGD_ERR_STATE, "a sharded state steps through bsgd_shard_begin / _end");
    if (n_iters > 0) BSGD_TRY(sync_xT(s, x, st));
    if (n_iters > 0 && s->iters == 0 && !s->zero_start) BSGD_TRY(warm_start(s, x, st));
    for (int k = 0; k < n_iters; ++k) BSGD_TRY(one_iteration(s, x, st, k > 0, k + 1 < n_iters));
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_state_query(bsgd_state *s, bsgd_report *out, void *stream) {
    if (!s || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = s->g->M * s->g->desc.nv;
    std::vector<double> S(n);
    unsigned long long upd = 0;
    BSGD_CUDA(cudaMemcpyAsync(S.data(), s->S, 8 * n, cudaMemcpyDeviceToHost, st));
    BSGD_CUDA(cudaMemcpyAsync(&upd, s->updates, 8, cudaMemcpyDeviceToHost, st));
    double mu = s->mu;
    BSGD_CUDA(cudaMemcpyAsync(&mu, s->d_mu, 8, cudaMemcpyDeviceToHost, st));
    BSGD_CUDA(cudaStreamSynchronize(st));
    double tot = 0.0;
    for (double v : S) tot += v;
    out->residual_norm = std::sqrt(std::max(tot, 0.0));
    out->mu = mu;
    out->iteration = s->iters;
    out->epoch = (double)s->iters / s->epoch_len;
    out->updates = (int64_t)upd;
    return BSGD_OK;
}

// ---------------------------------------------------------------------------
// Owner-computes sharding (Sec. 2, Fig. 1: the nodes hold column blocks x_J and
// the master sums their A_I^J x_J into r_I). Every process holds a state of the
// whole problem but computes only for the column blocks it owns; one iteration
// is bsgd_shard_begin (draw, FP of the owned drawn pairs, the process's part of
// sum_j z^j on the rows that changed), a sum of the exchange buffers over the
// processes (the caller's all-reduce), and bsgd_shard_end (r from the total, BP
// of the owned drawn pairs, update of the owned drawn blocks).

extern "C" bsgd_status bsgd_state_set_shard(bsgd_state *s, const int32_t *owned_blocks, int n_owned,
                                            int64_t *exchange_len) {
    if (!s || (!owned_blocks && n_owned > 0) || !exchange_len)
        return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (s->iters != 0) return fail(BSGD_ERR_STATE, "shard a state before its first iteration");
    if (s->p.pair_sampling != BSGD_PAIRS_UNIFORM || s->p.cells == BSGD_CELLS_GEOMETRIC ||
        s->p.tv_lambda > 0 || s->am || s->replay)
        return fail(BSGD_ERR_INVALID_ARG,
                    "sharded states draw uniform pairs (whole views or uniform cells), with no TV "
                    "prox, no automatic step and no replay");
    const bsgd_geometry *g = s->g;
    if (n_owned < 0 || n_owned > g->N) return fail(BSGD_ERR_INVALID_ARG, "n_owned out of range");
    std::vector<unsigned char> m(g->N, 0);
    for (int k = 0; k < n_owned; ++k) {
        if (owned_blocks[k] < 0 || owned_blocks[k] >= g->N)
            return fail(BSGD_ERR_INVALID_ARG, "owned block id out of range");
        m[owned_blocks[k]] = 1;
    }
    if (!s->owned) {
        BSGD_TRY(palloc((void **)&s->owned, g->N, 0));
        BSGD_CUDA(cudaStreamSynchronize(0));
    }
    BSGD_CUDA(cudaMemcpy(s->owned, m.data(), g->N, cudaMemcpyHostToDevice));
    s->dev.owned = s->owned;
    *exchange_len = (int64_t)s->kM * g->max_views * g->desc.nv * g->desc.nu;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_shard_begin(bsgd_state *s, void *x, float *exchange, void *stream) {
    if (!s || !x || !exchange) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!s->owned) return fail(BSGD_ERR_STATE, "not a sharded state (bsgd_state_set_shard)");
    BSGD_TRY(check_device(s->g));
    const bsgd_geometry *g = s->g;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t k = s->iters;
    if (k == 0 && !s->zero_start) {
        // the processes' memories start from x = 0 (a warm start would need
        // the sum of every process's A^j x0 first): refuse any other image
        int nz = 0;
        BSGD_TRY(launch_nonzero(g, x, s->st, s->x0_flag, st));
        BSGD_CUDA(cudaMemcpyAsync(&nz, s->x0_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        BSGD_CUDA(cudaStreamSynchronize(st));
        if (nz) return fail(BSGD_ERR_INVALID_ARG, "a sharded state starts from x = 0 on every process");
    }
    if (k == 0) BSGD_TRY(sync_xT(s, x, st));
    s->dev.work = work_buf(s, k);
    s->dev.cells = cells_buf(s, k);
    SampleArgs A;
    fill_sample_args(s, A, k);
    sample_kernel<<<1, kSampleThreads, 0, st>>>(A);
    BSGD_CUDA(cudaGetLastError());
    if (s->max_tiles > 0) BSGD_TRY(launch_fp_solve(g, s->dev, x, s->st, s->P, s->max_tiles, false, st));
    dim3 grid((g->desc.nv + kResRows - 1) / kResRows, g->max_views, s->kM);
    if (s->st == BSGD_F32) shard_partial_kernel<float><<<grid, 256, 0, st>>>(g->dg, s->dev, exchange);
    else if (s->st == BSGD_BF16) shard_partial_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(g->dg, s->dev, exchange);
    else shard_partial_kernel<__half><<<grid, 256, 0, st>>>(g->dg, s->dev, exchange);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_shard_end(bsgd_state *s, void *x, const float *exchange, void *stream) {
    if (!s || !x || !exchange) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!s->owned) return fail(BSGD_ERR_STATE, "not a sharded state (bsgd_state_set_shard)");
    const bsgd_geometry *g = s->g;
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid((g->desc.nv + kResRows - 1) / kResRows, g->max_views, s->kM);
    if (s->st == BSGD_F32) shard_residual_kernel<float><<<grid, 256, 0, st>>>(g->dg, s->dev, exchange);
    else if (s->st == BSGD_BF16) shard_residual_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(g->dg, s->dev, exchange);
    else shard_residual_kernel<__half><<<grid, 256, 0, st>>>(g->dg, s->dev, exchange);
    BSGD_CUDA(cudaGetLastError());
    if (s->max_tiles > 0) BSGD_TRY(launch_bp_solve(g, s->dev, s->st, s->P, s->max_tiles, st));
    BSGD_TRY(launch_update(s, x, st, false));
    s->iters += 1;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_state_read_residual(bsgd_state *s, void *out, bsgd_dtype ot,
                                                void *stream) {
    if (!s || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!dtype_ok(ot)) return fail(BSGD_ERR_INVALID_ARG, "bad dtype");
    return convert(s->r, s->st, out, ot, s->g->n_rows(), (cudaStream_t)stream);
}

extern "C" bsgd_status bsgd_state_profile(bsgd_state *s, int enable) {
    if (!s) return fail(BSGD_ERR_INVALID_ARG, "state is NULL");
    s->profiling = enable != 0;
    s->marks.clear();
    s->ev_used = 0;
    for (int k = 0; k < BSGD_N_STAGES; ++k) {
        s->launches[k] = 0;
        s->ms[k] = 0.0;
    }
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_state_set_sampling(bsgd_state *s, int pair_sampling, int cells,
                                               int n_cells, void *stream) {
    if (!s) return fail(BSGD_ERR_INVALID_ARG, "state is NULL");
    const bsgd_geometry *g = s->g;
    if (pair_sampling != BSGD_PAIRS_UNIFORM && pair_sampling != BSGD_PAIRS_RESIDUAL)
        return fail(BSGD_ERR_INVALID_ARG, "bad pair sampling");
    if (pair_sampling == BSGD_PAIRS_RESIDUAL && (s->P != 1 || g->M * g->N > kMaxResidualPairs))
        return fail(BSGD_ERR_INVALID_ARG, "residual pair sampling draws one pair per iteration");
    if (s->owned && (pair_sampling != BSGD_PAIRS_UNIFORM || cells == BSGD_CELLS_GEOMETRIC))
        return fail(BSGD_ERR_INVALID_ARG, "a sharded state draws uniform pairs and cells");
    if (cells < BSGD_CELLS_NONE || cells > BSGD_CELLS_UNIFORM)
        return fail(BSGD_ERR_INVALID_ARG, "bad cell sampling");
    if (cells != BSGD_CELLS_NONE && n_cells != (g->desc.nv > 1 ? 4 : 2))
        return fail(BSGD_ERR_INVALID_ARG, "n_cells must be 4 (3D) or 2 (2D)");
    const int nc = cells == BSGD_CELLS_NONE ? 1 : n_cells;
    unsigned long long *counts = nullptr;
    double *cw = nullptr;
    BSGD_TRY(geometry_tables(g, nc, cells == BSGD_CELLS_GEOMETRIC, (cudaStream_t)stream, &counts, &cw));
    s->p.pair_sampling = pair_sampling;
    s->p.cells = cells;
    s->p.n_cells = nc;
    s->n_cells = nc;
    s->counts = counts;
    s->cw = cw;
    s->dev.n_cells = nc;
    pair_updates_kernel<<<(g->M * g->N + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        g->dg, counts, nc, s->pair_upd);
    BSGD_CUDA(cudaGetLastError());
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_state_set_split(bsgd_state *s, int split) {
    if (!s) return fail(BSGD_ERR_INVALID_ARG, "state is NULL");
    s->split = split != 0;
    return BSGD_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: a header that identifies the state's shape, then the
// device arrays in a fixed order.

namespace {

struct CkptHeader {
    char magic[8];
    int32_t version, storage;
    int32_t kind, M, N, kM, kN, P;
    int32_t pair_sampling, cells, n_cells, auto_mu, has_tv, pad;
    int64_t nx, ny, nz, n_views, nu, nv;
    int64_t iters, trace_rows, payload;
    uint64_t seed;
};
constexpr char kCkptMagic[8] = {'B', 'S', 'G', 'D', 'C', 'K', 'P', 'T'};

struct CkptPart {
    void *dev;
    size_t bytes;
};

// The device arrays of a checkpoint, in blob order; trace rows = iterations
// recorded so far.
std::vector<CkptPart> ckpt_parts(const bsgd_state *s, int64_t trace_rows) {
    const bsgd_geometry *g = s->g;
    const size_t es = dtype_size(s->st), R = (size_t)g->n_rows(), C = (size_t)g->n_cols();
    const size_t Z = (size_t)g->zlen;
    std::vector<CkptPart> v = {
        {s->z, Z * es}, {s->rt, Z * es}, {s->r, R * es}, {s->grad, C * 4},
        {s->S, 8 * (size_t)g->M * g->desc.nv}, {s->d_mu, 8}, {s->d_iter, 8}, {s->updates, 8},
        {s->trace, 4 * (size_t)trace_rows * s->stride}};
    if (s->gT) v.push_back({s->gT, C * 4});
    if (s->xlo) v.push_back({s->xlo, C * es});
    if (s->eud) {
        v.push_back({s->eud, 8 * C});
        v.push_back({s->eud_prev, 8 * C});
        v.push_back({s->am, sizeof(AutoMuHist)});
    }
    return v;
}

CkptHeader ckpt_header(const bsgd_state *s) {
    const bsgd_geometry *g = s->g;
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.storage = s->st;
    h.kind = g->desc.kind;
    h.M = g->M;
    h.N = g->N;
    h.kM = s->kM;
    h.kN = s->kN;
    h.P = s->P;
    h.pair_sampling = s->p.pair_sampling;
    h.cells = s->p.cells;
    h.n_cells = s->n_cells;
    h.auto_mu = s->eud != nullptr;
    h.has_tv = s->p.tv_lambda > 0;
    h.nx = g->desc.nx, h.ny = g->desc.ny, h.nz = g->desc.nz;
    h.n_views = g->desc.n_views, h.nu = g->desc.nu, h.nv = g->desc.nv;
    h.iters = s->iters;
    h.trace_rows = std::min(s->iters, s->trace_cap);
    h.seed = s->p.seed;
    size_t tot = 0;
    for (const CkptPart &q : ckpt_parts(s, h.trace_rows)) tot += q.bytes;
    h.payload = (int64_t)tot;
    return h;
}

}  // namespace

extern "C" bsgd_status bsgd_state_checkpoint_bytes(const bsgd_state *s, int64_t *bytes) {
    if (!s || !bytes) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    *bytes = (int64_t)sizeof(CkptHeader) + ckpt_header(s).payload;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_state_save(bsgd_state *s, void *host, int64_t cap, void *stream) {
    if (!s || !host) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    const CkptHeader h = ckpt_header(s);
    if (cap < (int64_t)sizeof(CkptHeader) + h.payload)
        return fail(BSGD_ERR_INVALID_ARG, "checkpoint buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    char *out = static_cast<char *>(host);
    std::memcpy(out, &h, sizeof h);
    size_t off = sizeof h;
    for (const CkptPart &q : ckpt_parts(s, h.trace_rows)) {
        if (q.bytes) BSGD_CUDA(cudaMemcpyAsync(out + off, q.dev, q.bytes, cudaMemcpyDeviceToHost, st));
        off += q.bytes;
    }
    BSGD_CUDA(cudaStreamSynchronize(st));
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_state_restore(bsgd_state *s, const void *host, int64_t bytes,
                                          void *stream) {
    if (!s || !host) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (bytes < (int64_t)sizeof(CkptHeader)) return fail(BSGD_ERR_INVALID_ARG, "checkpoint truncated");
    CkptHeader h;
    std::memcpy(&h, host, sizeof h);
    const CkptHeader mine = ckpt_header(s);
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1)
        return fail(BSGD_ERR_INVALID_ARG, "not a BSGD checkpoint");
    if (h.storage != mine.storage || h.kind != mine.kind || h.M != mine.M || h.N != mine.N ||
        h.kM != mine.kM || h.kN != mine.kN || h.P != mine.P || h.auto_mu != mine.auto_mu ||
        h.has_tv != mine.has_tv || h.nx != mine.nx || h.ny != mine.ny || h.nz != mine.nz ||
        h.n_views != mine.n_views || h.nu != mine.nu || h.nv != mine.nv || h.seed != mine.seed)
        return fail(BSGD_ERR_INVALID_ARG, "checkpoint of a different geometry or solver set-up");
    if (h.iters < 0 || h.trace_rows != std::min(h.iters, s->trace_cap))
        return fail(BSGD_ERR_INVALID_ARG, "corrupt checkpoint header");
    const std::vector<CkptPart> parts = ckpt_parts(s, h.trace_rows);
    size_t need = 0;
    for (const CkptPart &q : parts) need += q.bytes;
    if ((int64_t)need != h.payload || bytes < (int64_t)sizeof(CkptHeader) + h.payload)
        return fail(BSGD_ERR_INVALID_ARG, "checkpoint truncated");
    cudaStream_t st = (cudaStream_t)stream;
    if (h.pair_sampling != s->p.pair_sampling || h.cells != s->p.cells || h.n_cells != s->n_cells)
        BSGD_TRY(bsgd_state_set_sampling(s, h.pair_sampling, h.cells, h.n_cells, stream));
    const char *in = static_cast<const char *>(host) + sizeof h;
    for (const CkptPart &q : parts) {
        if (q.bytes) BSGD_CUDA(cudaMemcpyAsync(q.dev, in, q.bytes, cudaMemcpyHostToDevice, st));
        in += q.bytes;
    }
    BSGD_CUDA(cudaStreamSynchronize(st));
    s->iters = h.iters;
    cudaFree(s->replay);   // a replay in progress belongs to the state that was replaced
    s->replay = nullptr;
    s->replay_n = 0;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_state_read_profile(bsgd_state *s, bsgd_profile *out, void *stream) {
    if (!s || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    BSGD_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    for (auto &m : s->marks) {
        float t = 0.f;
        BSGD_CUDA(cudaEventElapsedTime(&t, m.second.first, m.second.second));
        s->ms[m.first] += t;
    }
    s->marks.clear();
    s->ev_used = 0;
    for (int k = 0; k < BSGD_N_STAGES; ++k) {
        out->launches[k] = s->launches[k];
        out->ms[k] = s->ms[k];
    }
    return BSGD_OK;
}

extern "C" int64_t bsgd_trace_stride(const bsgd_state *s) { return s ? s->stride : 0; }

extern "C" bsgd_status bsgd_state_read_trace(bsgd_state *s, int32_t *host, int64_t cap,
                                             int64_t n_iters, void *stream) {
    if (!s || !host) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (n_iters < 0 || n_iters > s->iters || n_iters > s->trace_cap)
        return fail(BSGD_ERR_INVALID_ARG, "n_iters beyond the recorded iterations");
    if (n_iters * s->stride > cap) return fail(BSGD_ERR_INVALID_ARG, "host buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    BSGD_CUDA(cudaMemcpyAsync(host, s->trace, 4 * n_iters * s->stride, cudaMemcpyDeviceToHost, st));
    BSGD_CUDA(cudaStreamSynchronize(st));
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_state_set_replay(bsgd_state *s, const int32_t *host, int64_t n_iters) {
    if (!s || (!host && n_iters > 0)) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (s->owned && n_iters > 0) return fail(BSGD_ERR_INVALID_ARG, "a sharded state replays no trace");
    if (n_iters < 0) return fail(BSGD_ERR_INVALID_ARG, "n_iters < 0");
    const bsgd_geometry *g = s->g;
    for (int64_t t = 0; t < n_iters; ++t) {
        const int32_t *e = host + t * s->stride;
        if (e[0] < 1 || e[0] > s->P) return fail(BSGD_ERR_INVALID_ARG, "bad pair count in trace");
        for (int p = 0; p < e[0]; ++p) {
            if (e[1 + 2 * p] < 0 || e[1 + 2 * p] >= g->M || e[2 + 2 * p] < 0 || e[2 + 2 * p] >= g->N)
                return fail(BSGD_ERR_INVALID_ARG, "block id out of range in trace");
            for (int k = 0; k < g->max_views; ++k) {
                const int c = e[1 + 2 * e[0] + p * g->max_views + k];
                if (c < -1 || c >= s->n_cells || (c == -1 && s->p.cells != BSGD_CELLS_NONE &&
                                                  k < (int)g->block_views[e[1 + 2 * p]].size()))
                    return fail(BSGD_ERR_INVALID_ARG, "bad cell id in trace");
            }
        }
    }
    cudaDeviceSynchronize();
    cudaFree(s->replay);
    s->replay = nullptr;
    s->replay_n = 0;
    if (n_iters > 0) BSGD_TRY(upload((void **)&s->replay, host, 4 * n_iters * s->stride));
    s->replay_start = s->iters;
    s->replay_n = n_iters;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_solve(const bsgd_geometry *g, const bsgd_solve_params *p,
                                  const void *y, bsgd_dtype yt, void *x, bsgd_dtype xt,
                                  bsgd_report *out, void *stream) {
    if (!g || !p || !y || !x) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!dtype_ok(yt) || !dtype_ok(xt)) return fail(BSGD_ERR_INVALID_ARG, "bad dtype");
    BSGD_TRY(check_device(g));
    cudaStream_t st = (cudaStream_t)stream;
    auto on_host = [](const void *ptr) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            cudaGetLastError();
            return true;
        }
        return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
    };
    const int64_t R = g->n_rows(), C = g->n_cols();
    const bool yh = on_host(y), xh = on_host(x);
    void *dy = nullptr, *dx = nullptr, *xs = nullptr;
    bsgd_state *s = nullptr;
    bsgd_status e = BSGD_OK;
    auto body = [&]() -> bsgd_status {
        const void *yy = y;
        if (yh) {
            BSGD_TRY(palloc(&dy, R * dtype_size(yt), st));
            BSGD_CUDA(cudaMemcpyAsync(dy, y, R * dtype_size(yt), cudaMemcpyHostToDevice, st));
            yy = dy;
        }
        BSGD_TRY(bsgd_state_create(g, p, yy, yt, stream, &s));
        const bsgd_dtype sd = (bsgd_dtype)p->storage;
        BSGD_TRY(palloc(&xs, C * dtype_size(sd), st));
        // x holds the starting image x0 (the first block step warm-starts from
        // it) unless the caller asks for Algorithm 1's zero start
        if (xh) BSGD_TRY(palloc(&dx, C * dtype_size(xt), st));
        if (p->zero_start) {
            BSGD_CUDA(cudaMemsetAsync(xs, 0, C * dtype_size(sd), st));
            s->zero_start = true;   // the state already describes x0 = 0
        } else {
            const void *x0 = x;
            if (xh) {
                BSGD_CUDA(cudaMemcpyAsync(dx, x, C * dtype_size(xt), cudaMemcpyHostToDevice, st));
                x0 = dx;
            }
            BSGD_TRY(convert(x0, xt, xs, sd, C, st));
        }
        const int fin = std::max(0, std::min(p->final_uniform_epochs, p->epochs));
        BSGD_TRY(bsgd_block_step(s, xs, (p->epochs - fin) * s->epoch_len, stream));
        if (fin > 0) {   // last epochs without importance sampling (after Algorithm 2)
            BSGD_TRY(bsgd_state_set_sampling(s, BSGD_PAIRS_UNIFORM, BSGD_CELLS_NONE, 1, stream));
            BSGD_TRY(bsgd_block_step(s, xs, fin * s->epoch_len, stream));
        }
        void *xo = xh ? dx : x;
        BSGD_TRY(convert(xs, sd, xo, xt, C, st));
        if (xh) BSGD_CUDA(cudaMemcpyAsync(x, dx, C * dtype_size(xt), cudaMemcpyDeviceToHost, st));
        if (out) BSGD_TRY(bsgd_state_query(s, out, stream));
        BSGD_CUDA(cudaStreamSynchronize(st));
        return BSGD_OK;
    };
    e = body();
    cudaStreamSynchronize(st);
    if (s) bsgd_state_destroy(s);
    pfree(dy);
    pfree(dx);
    pfree(xs);
    return e;
}
