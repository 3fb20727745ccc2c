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
//   K6c k_gftt_sort   one CTA, bitonic sort of the keys, descending.
//   K6d k_gftt_greedy one warp: candidates in priority order, 32 at a time;
//                     each lane checks its candidate against the kept corners
//                     through a cell grid in shared memory (cells at least
//                     min_dist wide, linked lists), then the 32 are resolved
//                     in order by warp votes; stops at max_corners.
// Every decision is taken on the same FP32 values the oracle computes, so the
// corner list is exact.
#include <cstdint>
#include <cstdlib>

#include "vt_internal.cuh"

namespace vt {

constexpr int GF_BX = 32, GF_BY = 8;
constexpr int GF_SORT_THREADS = 1024;
constexpr int GF_MAX_CELLS = 24576;     // cell-grid heads in shared memory (int16)
constexpr int GF_MAX_CORNERS = 8192;

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

// Bitonic sort (descending) of the first `n` keys, padded with zeros to a power of two.
__global__ void __launch_bounds__(GF_SORT_THREADS) k_gftt_sort(unsigned long long *keys, const int *count, int cap) {
    const int n = min(*count, cap);
    int N = 1;
    while (N < n) N <<= 1;
    for (int i = n + threadIdx.x; i < N; i += blockDim.x) keys[i] = 0ull;
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const int p = i ^ j;
                if (p > i) {
                    const unsigned long long a = keys[i], b = keys[p];
                    const bool desc = (i & k) == 0;
                    if (desc ? (a < b) : (a > b)) {
                        keys[i] = b;
                        keys[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void k_gftt_greedy(const unsigned long long *keys, const int *count, int cap, int w, int h, int min_dist,
                              int cell, int cells_x, int cells_y, int max_corners, float2 *out, float *out_score,
                              int *out_count) {
    extern __shared__ __align__(16) uint8_t gf_smem[];
    int16_t *head = reinterpret_cast<int16_t *>(gf_smem);                 // [cells_x * cells_y]
    int16_t *next = head + ((cells_x * cells_y + 7) & ~7);                // [max_corners]
    uint32_t *kxy = reinterpret_cast<uint32_t *>(next + ((max_corners + 7) & ~7));  // [max_corners]
    const int lane = threadIdx.x;
    const int ncell = cells_x * cells_y;
    for (int i = lane; i < ncell; i += 32) head[i] = -1;
    __syncwarp();
    const int n = min(*count, cap);
    const long d2 = (long)min_dist * min_dist;
    int kept = 0;
    for (int base = 0; base < n && kept < max_corners; base += 32) {
        const int i = base + lane;
        const bool have = i < n;
        unsigned long long key = have ? keys[i] : 0ull;
        const unsigned idx = 0xffffffffu - (unsigned)(key & 0xffffffffu);
        const int x = have ? (int)(idx % (unsigned)w) : 0, y = have ? (int)(idx / (unsigned)w) : 0;
        bool ok = have;
        if (ok) {  // against the corners kept by earlier chunks
            const int cx = x / cell, cy = y / cell;
            for (int dy = -1; dy <= 1 && ok; ++dy) {
                const int yy = cy + dy;
                if (yy < 0 || yy >= cells_y) continue;
                for (int dx = -1; dx <= 1 && ok; ++dx) {
                    const int xx = cx + dx;
                    if (xx < 0 || xx >= cells_x) continue;
                    for (int e = head[yy * cells_x + xx]; e >= 0; e = next[e]) {
                        const uint32_t p = kxy[e];
                        const long ex = (long)(p & 0xffffu) - x, ey = (long)(p >> 16) - y;
                        if (ex * ex + ey * ey < d2) {
                            ok = false;
                            break;
                        }
                    }
                }
            }
        }
        // resolve the chunk in priority order
        for (int j = 0; j < 32 && kept < max_corners; ++j) {
            const unsigned okmask = __ballot_sync(0xffffffffu, ok);
            if (!((okmask >> j) & 1u)) continue;
            const int xj = __shfl_sync(0xffffffffu, x, j), yj = __shfl_sync(0xffffffffu, y, j);
            if (lane > j && ok) {
                const long ex = (long)x - xj, ey = (long)y - yj;
                if (ex * ex + ey * ey < d2) ok = false;
            }
            if (lane == j) {
                const int c = (y / cell) * cells_x + (x / cell);
                kxy[kept] = (uint32_t)x | ((uint32_t)y << 16);
                next[kept] = head[c];
                head[c] = (int16_t)kept;
                out[kept] = make_float2((float)x, (float)y);
                if (out_score) out_score[kept] = __uint_as_float((unsigned)(key >> 32));
            }
            __syncwarp();
            ++kept;
        }
    }
    if (lane == 0) *out_count = kept;
}

}  // namespace vt

using namespace vt;

struct vt_gftt {
    int max_w, max_h;
    float *score;
    unsigned *maxbits;  // [1], followed by the candidate count
    int *count;
    unsigned long long *keys;
    int cap;
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
    bool ok = cudaMalloc(&g->score, sizeof(float) * (size_t)max_w * max_h) == cudaSuccess &&
              cudaMalloc(&g->maxbits, 2 * sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&g->keys, sizeof(unsigned long long) * (size_t)N) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        vt_gftt_free(g);
        return VT_ERR_OOM;
    }
    g->count = reinterpret_cast<int *>(g->maxbits + 1);
    *out = g;
    return VT_OK;
}

void vt_gftt_free(vt_gftt *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->score) cudaFree(g->score);
    if (g->maxbits) cudaFree(g->maxbits);
    if (g->keys) cudaFree(g->keys);
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
    // cells at least min_dist wide, few enough for the shared-memory heads
    int cell = prm->min_dist;
    while ((long)((L.w + cell - 1) / cell) * ((L.h + cell - 1) / cell) > GF_MAX_CELLS) ++cell;
    const int cx = (L.w + cell - 1) / cell, cy = (L.h + cell - 1) / cell;
    const size_t smem = sizeof(int16_t) * (((size_t)cx * cy + 7) & ~(size_t)7) +
                        sizeof(int16_t) * ((prm->max_corners + 7) & ~7) + sizeof(uint32_t) * prm->max_corners;
    if (cudaMemsetAsync(g->maxbits, 0, 2 * sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    const dim3 blk(GF_BX, GF_BY), grd((L.w + GF_BX - 1) / GF_BX, (L.h + GF_BY - 1) / GF_BY);
    k_gftt_score<<<grd, blk, 0, s>>>(L.grad, L.gpitch, L.w, L.h, prm->block_radius, g->score, g->maxbits);
    k_gftt_cand<<<grd, blk, 0, s>>>(g->score, L.w, L.h, g->maxbits, prm->quality, prm->nms_radius, prm->border,
                                    reinterpret_cast<const float2 *>(mask_pts), n_mask, prm->min_dist, g->keys,
                                    g->count, g->cap);
    k_gftt_sort<<<1, GF_SORT_THREADS, 0, s>>>(g->keys, g->count, g->cap);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gftt_greedy, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        attr = true;
    }
    k_gftt_greedy<<<1, 32, smem, s>>>(g->keys, g->count, g->cap, L.w, L.h, prm->min_dist, cell, cx, cy,
                                      prm->max_corners, reinterpret_cast<float2 *>(corners_out), scores_out,
                                      count_out);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

}  // extern "C"
