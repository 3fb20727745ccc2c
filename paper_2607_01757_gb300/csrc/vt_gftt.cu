// Shi-Tomasi (GFTT) corner detection on a pyramid level (the classical
// detector the paper pairs with LK tracking, Sec. IV; run on the CPU in the
// paper, Sec. V-F).  It reuses the level's stored Scharr gradients.
//
//   K6a k_gftt_score  a, b, c = (2br+1)^2 box sums of gx^2, gx gy, gy^2
//                     (exact integers), lambda_min in FP32 with explicit
//                     round-to-nearest operations, clamped at 0; the block
//                     maxima go to one atomic maximum.
//   K6b k_gftt_cand   lambda >= quality * max, lambda > 0, outside the border,
//                     local maximum of its (2nms+1)^2 neighbourhood (ties to
//                     the smaller index), far enough from every mask point:
//                     appended as a 64-bit key (score bits, ~index).
//   K6c cell grid     counting sort of the candidates into cells at least
//                     min_dist wide (count, one-CTA scan, scatter).
//   K6d k_gftt_select the greedy min-distance selection in priority order,
//                     resolved in parallel rounds over the cell grid
//                     (cooperative launch, grid-wide barrier per round).
//   K6e k_gftt_output the kept candidates sorted (shared-memory bitonic sort)
//                     and the first max_corners written out.
// Every decision is taken on the same FP32 values the oracle computes, so the
// corner list is exact.
#include <cooperative_groups.h>

#include <cstdint>
#include <cstdlib>

#include "vt_internal.cuh"

namespace cg = cooperative_groups;

namespace vt {

constexpr int GF_BX = 32, GF_BY = 8;
constexpr int GF_SORT_THREADS = 1024;
constexpr int GF_SCAN_THREADS = 1024;
constexpr int GF_MIS_THREADS = 256;
constexpr int GF_SMEM_SORT = 16384;  // kept keys sorted in shared memory (128 KB)
constexpr int GF_MAX_CORNERS = 8192;
constexpr int GF_GRID_THREADS = 256;
enum : uint8_t { GF_UNDECIDED = 0, GF_KEPT = 1, GF_REJECTED = 2 };

__device__ __forceinline__ float gftt_score(long long a, long long b, long long c) {
    const float fa = (float)a, fb = (float)b, fc = (float)c;
    const float d = __fsub_rn(fa, fc);
    const float q = __fadd_rn(__fmul_rn(d, d), __fmul_rn(4.0f, __fmul_rn(fb, fb)));
    const float t = __fsub_rn(__fadd_rn(fa, fc), __fsqrt_rn(q));
    const float l = __fmul_rn(0.5f, t);
    return l > 0.0f ? l : 0.0f;
}

__global__ void k_gftt_score(const uint32_t *grad, int gpitch, int w, int h, int br, float *score,
                             unsigned *maxbits) {
    const int x = blockIdx.x * GF_BX + threadIdx.x, y = blockIdx.y * GF_BY + threadIdx.y;
    float s = 0.0f;
    if (x < w && y < h) {
        long long a = 0, b = 0, c = 0;
        for (int j = -br; j <= br; ++j) {
            const uint32_t *row = grad + (size_t)refl101(y + j, h) * gpitch;
            for (int i = -br; i <= br; ++i) {
                const uint32_t v = __ldg(row + refl101(x + i, w));
                const long long u = (int16_t)(v & 0xffffu), t = (int16_t)(v >> 16);
                a += u * u;
                b += u * t;
                c += t * t;
            }
        }
        s = gftt_score(a, b, c);
        score[(size_t)y * w + x] = s;
    }
    // block maximum (scores are >= 0, so their bit patterns order like the values)
    unsigned m = __float_as_uint(s);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ unsigned wm[GF_BX * GF_BY / 32];
    const int tid = threadIdx.y * GF_BX + threadIdx.x;
    if ((tid & 31) == 0) wm[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        unsigned mm = 0;
        for (int k = 0; k < GF_BX * GF_BY / 32; ++k) mm = max(mm, wm[k]);
        atomicMax(maxbits, mm);
    }
}

__global__ void k_gftt_cand(const float *score, int w, int h, const unsigned *maxbits, float quality, int nms,
                            int border, const float2 *mask, int n_mask, int min_dist, unsigned long long *keys,
                            int *count, int cap) {
    const int x = blockIdx.x * GF_BX + threadIdx.x, y = blockIdx.y * GF_BY + threadIdx.y;
    if (x < border || y < border || x >= w - border || y >= h - border) return;
    const long idx = (long)y * w + x;
    const float s = score[idx];
    const float thr = __fmul_rn(quality, __uint_as_float(*maxbits));
    if (!(s >= thr) || !(s > 0.0f)) return;
    for (int j = -nms; j <= nms; ++j) {
        const int yy = y + j;
        if (yy < 0 || yy >= h) continue;
        for (int i = -nms; i <= nms; ++i) {
            const int xx = x + i;
            if ((i == 0 && j == 0) || xx < 0 || xx >= w) continue;
            const long q = (long)yy * w + xx;
            const float t = score[q];
            if (t > s || (t == s && q < idx)) return;
        }
    }
    const float md2 = (float)(min_dist * min_dist);
    for (int m = 0; m < n_mask; ++m) {
        const float2 p = mask[m];
        const float dx = __fsub_rn((float)x, p.x), dy = __fsub_rn((float)y, p.y);
        if (__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) < md2) return;
    }
    const int slot = atomicAdd(count, 1);
    if (slot < cap)
        keys[slot] = ((unsigned long long)__float_as_uint(s) << 32) | (unsigned long long)(0xffffffffu - (unsigned)idx);
}

__device__ __forceinline__ unsigned key_index(unsigned long long k) { return 0xffffffffu - (unsigned)(k & 0xffffffffu); }

// Candidates into a grid of cells at least min_dist wide (a counting sort:
// count, scan, scatter), so every pair closer than min_dist lies in
// neighbouring cells.
__global__ void k_gftt_cell_count(const unsigned long long *keys, const int *count, int cap, int w, int cell,
                                  int cells_x, int *cell_count, int *rank) {
    const int n = min(*count, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned idx = key_index(keys[i]);
        const int x = (int)(idx % (unsigned)w), y = (int)(idx / (unsigned)w);
        rank[i] = atomicAdd(&cell_count[(y / cell) * cells_x + x / cell], 1);
    }
}

// Exclusive scan of cell_count[0..ncell) into cell_start[0..ncell] (one CTA).
__global__ void __launch_bounds__(GF_SCAN_THREADS) k_gftt_cell_scan(const int *cell_count, int ncell,
                                                                      int *cell_start) {
    __shared__ int part[GF_SCAN_THREADS];
    const int per = (ncell + GF_SCAN_THREADS - 1) / GF_SCAN_THREADS;
    const int b = threadIdx.x * per, e = min(ncell, b + per);
    int sum = 0;
    for (int i = b; i < e; ++i) sum += cell_count[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < GF_SCAN_THREADS; o <<= 1) {  // inclusive Hillis-Steele scan of the partial sums
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - sum;
    for (int i = b; i < e; ++i) {
        cell_start[i] = run;
        run += cell_count[i];
    }
    if (threadIdx.x == GF_SCAN_THREADS - 1) cell_start[ncell] = part[GF_SCAN_THREADS - 1];
}

__global__ void k_gftt_cell_scatter(const unsigned long long *keys, const int *count, int cap, int w, int cell,
                                    int cells_x, const int *cell_start, const int *rank, unsigned long long *skeys,
                                    uint8_t *state) {
    const int n = min(*count, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        const unsigned idx = key_index(k);
        const int x = (int)(idx % (unsigned)w), y = (int)(idx / (unsigned)w);
        const int pos = cell_start[(y / cell) * cells_x + x / cell] + rank[i];
        skeys[pos] = k;
        state[pos] = GF_UNDECIDED;
    }
}

// The greedy min-distance selection, resolved in parallel rounds.  In
// priority order, a candidate is kept when no kept candidate lies closer than
// min_dist; its fate therefore depends only on the higher-priority
// candidates within min_dist.  Each round decides every undecided candidate
// whose closer higher-priority neighbours are all decided: rejected if one of
// them is kept, kept otherwise.  States only move from undecided to final,
// and a final state is the sequential greedy's, so reading a neighbour that
// another thread finalises in the same round is harmless.  The highest-
// priority undecided candidate is always decided, so the rounds end (in
// practice after a few dozen).  Rounds are separated by grid-wide barriers
// (cooperative launch); the kept candidates are then appended to `kept`.
__global__ void __launch_bounds__(GF_MIS_THREADS) k_gftt_select(const unsigned long long *skeys, const int *count,
                                                                 int cap, int w, int cell, int cells_x, int cells_y,
                                                                 const int *cell_start, uint8_t *state, int *und,
                                                                 long long d2, unsigned long long *kept,
                                                                 int *kept_count) {
    cg::grid_group grid = cg::this_grid();
    const int n = min(*count, cap);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    volatile uint8_t *vs = state;
    for (int r = 0;; ++r) {
        if (tid == 0) und[(r + 1) % 3] = 0;  // the slot round r+1 counts into (last read before round r)
        int mine = 0;
        for (int i = tid; i < n; i += nth) {
            if (vs[i] != GF_UNDECIDED) continue;
            const unsigned long long k = skeys[i];
            const unsigned idx = key_index(k);
            const int x = (int)(idx % (unsigned)w), y = (int)(idx / (unsigned)w);
            const int cx = x / cell, cy = y / cell;
            bool blocked = false, rejected = false;
            for (int dy = -1; dy <= 1 && !rejected; ++dy) {
                const int yy = cy + dy;
                if (yy < 0 || yy >= cells_y) continue;
                for (int dx = -1; dx <= 1 && !rejected; ++dx) {
                    const int xx = cx + dx;
                    if (xx < 0 || xx >= cells_x) continue;
                    const int c = yy * cells_x + xx;
                    for (int j = cell_start[c], je = cell_start[c + 1]; j < je; ++j) {
                        const unsigned long long kj = skeys[j];
                        if (kj <= k) continue;  // lower priority (or itself)
                        const unsigned jdx = key_index(kj);
                        const long long ex = (long long)(int)(jdx % (unsigned)w) - x;
                        const long long ey = (long long)(int)(jdx / (unsigned)w) - y;
                        if (ex * ex + ey * ey >= d2) continue;
                        const uint8_t sj = vs[j];
                        if (sj == GF_KEPT) {
                            rejected = true;
                            break;
                        }
                        if (sj == GF_UNDECIDED) blocked = true;
                    }
                }
            }
            if (rejected) vs[i] = GF_REJECTED;
            else if (!blocked) vs[i] = GF_KEPT;
            else ++mine;
        }
        if (mine) atomicAdd(&und[r % 3], mine);
        grid.sync();
        if (*reinterpret_cast<volatile int *>(&und[r % 3]) == 0) break;
    }
    for (int i = tid; i < n; i += nth)
        if (vs[i] == GF_KEPT) kept[atomicAdd(kept_count, 1)] = skeys[i];
}

// Kept candidates in priority order (keys descending), the first max_corners
// written out.  Up to GF_SMEM_SORT keys are sorted in shared memory; more
// (very large levels with a small min_dist) fall back to a bitonic sort in
// global memory (keys padded to a power of two <= kept capacity).
__global__ void __launch_bounds__(GF_SORT_THREADS) k_gftt_output(unsigned long long *kept, const int *kept_count,
                                                                  int kept_cap, int w, int max_corners, float2 *out,
                                                                  float *out_score, int *out_count) {
    extern __shared__ __align__(16) unsigned long long sk[];
    const int K = *kept_count;
    int N = 1;
    while (N < K) N <<= 1;
    const bool in_smem = N <= GF_SMEM_SORT;
    unsigned long long *a = in_smem ? sk : kept;
    if (in_smem)
        for (int i = threadIdx.x; i < N; i += blockDim.x) sk[i] = i < K ? kept[i] : 0ull;
    else
        for (int i = K + threadIdx.x; i < N && i < kept_cap; i += blockDim.x) kept[i] = 0ull;
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const int p = i ^ j;
                if (p > i) {
                    const unsigned long long x = a[i], y = a[p];
                    const bool desc = (i & k) == 0;
                    if (desc ? (x < y) : (x > y)) {
                        a[i] = y;
                        a[p] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int m = min(K, max_corners);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const unsigned long long k = a[i];
        const unsigned idx = key_index(k);
        out[i] = make_float2((float)(idx % (unsigned)w), (float)(idx / (unsigned)w));
        if (out_score) out_score[i] = __uint_as_float((unsigned)(k >> 32));
    }
    if (threadIdx.x == 0) *out_count = m;
}

}  // namespace vt

using namespace vt;

struct vt_gftt {
    int max_w, max_h;
    float *score;
    int *counters;  // [0] max score bits, [1] candidates, [2] kept, [3..5] undecided per round (3 slots)
    unsigned long long *keys;   // candidates (unordered); reused for the kept keys
    unsigned long long *skeys;  // candidates grouped by cell
    int *rank;
    uint8_t *state;
    int *cell_count, *cell_start;
    int cap, keys_cap;  // candidate capacity (pixels), keys buffer (power of two >= cap)
    int sms, select_grid;
};

extern "C" {

vt_status vt_gftt_create(int max_w, int max_h, vt_gftt **out) {
    if (!out || max_w <= 0 || max_h <= 0 || max_w > 65535 || max_h > 65535) return VT_ERR_ARG;
    vt_gftt *g = (vt_gftt *)calloc(1, sizeof(vt_gftt));
    if (!g) return VT_ERR_OOM;
    g->max_w = max_w;
    g->max_h = max_h;
    g->cap = max_w * max_h;
    int N = 1;
    while (N < g->cap) N <<= 1;
    g->keys_cap = N;
    const size_t px = (size_t)max_w * max_h;
    bool ok = cudaMalloc(&g->score, sizeof(float) * px) == cudaSuccess &&
              cudaMalloc(&g->counters, 8 * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&g->keys, sizeof(unsigned long long) * (size_t)N) == cudaSuccess &&
              cudaMalloc(&g->skeys, sizeof(unsigned long long) * px) == cudaSuccess &&
              cudaMalloc(&g->rank, sizeof(int) * px) == cudaSuccess &&
              cudaMalloc(&g->state, px) == cudaSuccess &&
              cudaMalloc(&g->cell_count, sizeof(int) * (px + 1)) == cudaSuccess &&
              cudaMalloc(&g->cell_start, sizeof(int) * (px + 1)) == cudaSuccess;
    int dev = 0, occ = 0;
    ok = ok && cudaGetDevice(&dev) == cudaSuccess &&
         cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
         cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gftt_select, GF_MIS_THREADS, 0) == cudaSuccess;
    if (!ok || occ < 1) {
        cudaGetLastError();
        vt_gftt_free(g);
        return ok ? VT_ERR_CUDA : VT_ERR_OOM;
    }
    g->select_grid = g->sms * (occ < 2 ? occ : 2);  // co-resident by construction (cooperative launch)
    *out = g;
    return VT_OK;
}

void vt_gftt_free(vt_gftt *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    cudaFree(g->score);
    cudaFree(g->counters);
    cudaFree(g->keys);
    cudaFree(g->skeys);
    cudaFree(g->rank);
    cudaFree(g->state);
    cudaFree(g->cell_count);
    cudaFree(g->cell_start);
    free(g);
}

vt_status vt_gftt_detect(vt_gftt *g, const vt_pyramid *p, int level, const vt_gftt_params *prm, const float *mask_pts,
                         int n_mask, float *corners_out, float *scores_out, int *count_out, void *cuda_stream) {
    if (!g || !p || !prm || !corners_out || !count_out) return VT_ERR_ARG;
    if (level < 0 || level >= p->levels || p->gtype != VT_GRAD_S16) return VT_ERR_ARG;
    const Level &L = p->lv[level];
    if (L.w > g->max_w || L.h > g->max_h) return VT_ERR_ARG;
    if (prm->max_corners < 0 || prm->max_corners > GF_MAX_CORNERS || !(prm->quality >= 0.f) ||
        prm->min_dist < 1 || prm->nms_radius < 0 || prm->block_radius < 0 || prm->block_radius > 3 ||
        prm->border < 0 || n_mask < 0 || (n_mask > 0 && !mask_pts))
        return VT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int cell = prm->min_dist;  // cells at least min_dist wide: close pairs are in neighbouring cells
    const int cx = (L.w + cell - 1) / cell, cy = (L.h + cell - 1) / cell, ncell = cx * cy;
    int *maxbits = g->counters, *count = g->counters + 1, *kept_count = g->counters + 2, *und = g->counters + 3;
    if (cudaMemsetAsync(g->counters, 0, 8 * sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(g->cell_count, 0, sizeof(int) * (size_t)ncell, s) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gftt_output, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(GF_SMEM_SORT * sizeof(unsigned long long)));
        attr = true;
    }
    const dim3 blk(GF_BX, GF_BY), grd((L.w + GF_BX - 1) / GF_BX, (L.h + GF_BY - 1) / GF_BY);
    k_gftt_score<<<grd, blk, 0, s>>>(L.grad, L.gpitch, L.w, L.h, prm->block_radius, g->score,
                                     reinterpret_cast<unsigned *>(maxbits));
    k_gftt_cand<<<grd, blk, 0, s>>>(g->score, L.w, L.h, reinterpret_cast<const unsigned *>(maxbits), prm->quality,
                                    prm->nms_radius, prm->border, reinterpret_cast<const float2 *>(mask_pts), n_mask,
                                    prm->min_dist, g->keys, count, g->cap);
    const int gg = 4 * g->sms;
    k_gftt_cell_count<<<gg, GF_GRID_THREADS, 0, s>>>(g->keys, count, g->cap, L.w, cell, cx, g->cell_count, g->rank);
    k_gftt_cell_scan<<<1, GF_SCAN_THREADS, 0, s>>>(g->cell_count, ncell, g->cell_start);
    k_gftt_cell_scatter<<<gg, GF_GRID_THREADS, 0, s>>>(g->keys, count, g->cap, L.w, cell, cx, g->cell_start, g->rank,
                                                       g->skeys, g->state);
    {
        const unsigned long long *skeys = g->skeys;
        const int *cell_start = g->cell_start;
        uint8_t *state = g->state;
        unsigned long long *kept = g->keys;
        int cap = g->cap, w = L.w;
        long long d2 = (long long)prm->min_dist * prm->min_dist;
        void *args[] = {(void *)&skeys, (void *)&count, (void *)&cap,   (void *)&w,          (void *)&cell,
                        (void *)&cx,    (void *)&cy,    (void *)&cell_start, (void *)&state, (void *)&und,
                        (void *)&d2,    (void *)&kept,  (void *)&kept_count};
        if (cudaLaunchCooperativeKernel((const void *)k_gftt_select, g->select_grid, GF_MIS_THREADS, args, 0, s) !=
            cudaSuccess) {
            cudaGetLastError();
            return VT_ERR_CUDA;
        }
    }
    k_gftt_output<<<1, GF_SORT_THREADS, GF_SMEM_SORT * sizeof(unsigned long long), s>>>(
        g->keys, kept_count, g->keys_cap, L.w, prm->max_corners, reinterpret_cast<float2 *>(corners_out), scores_out,
        count_out);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

}  // extern "C"
