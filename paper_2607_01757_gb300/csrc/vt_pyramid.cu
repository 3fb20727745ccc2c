// Gaussian pyramid (K1) and Scharr gradients (K2) for the LK tracker.
//
// K1: level l+1 = 5x5 separable [1 4 6 4 1]^2 / 256 sum centred at (2x, 2y)
//     of level l, reflect-101 borders, (s + 128) >> 8.  Integer arithmetic,
//     no rounding between the vertical and horizontal passes: bit-exact.
// K2: Scharr dx = [-3 0 3; -10 0 10; -3 0 3] * I, dy = transpose, reflect-101,
//     stored as (dx, dy) int16 pairs or (dx/32, dy/32) half pairs.
// The paper names the pyramidal LK tracker without its filters (Sec. IV,
// Table I); these are the readings implemented.
//
// Layout: a CTA stages its input tile (plus halo) in shared memory with
// 16-byte vector loads when the tile is inside the image, or with
// reflect-101 index mapping byte by byte on border tiles.  The same staged
// tile serves the pyramid step and, in the fused variant, the gradients of
// the source level.  Several levels / frames run in one launch through a
// job table passed as a __grid_constant__ kernel parameter.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "vt_internal.cuh"

namespace vt {

constexpr int PD_TW = 64;              // output tile width (level l+1)
constexpr int PD_TH = 16;              // output tile height
constexpr int PD_IW = 2 * PD_TW + 32;  // staged bytes per row (16-byte chunks)
constexpr int PD_IH = 2 * PD_TH + 3;   // staged rows
constexpr int PD_VW = 2 * PD_TW + 4;   // vertical-pass columns
constexpr int PD_THREADS = 256;

constexpr int SC_TW = 64;
constexpr int SC_TH = 16;
constexpr int SC_IW = SC_TW + 32;
constexpr int SC_IH = SC_TH + 2;
constexpr int SC_THREADS = 256;

template <int GT>
__device__ __forceinline__ uint32_t pack_grad(int dx, int dy) {
    if (GT == VT_GRAD_S16) {
        return (uint32_t)(uint16_t)(int16_t)dx | ((uint32_t)(uint16_t)(int16_t)dy << 16);
    } else {
        // raw / 32 is exact in FP32; the conversion to half rounds to nearest even
        __half2 h = __floats2half2_rn((float)dx * 0.03125f, (float)dy * 0.03125f);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

// Scharr of the staged tile at staged (row sr, column sc).
template <int IW>
__device__ __forceinline__ void scharr_at(const uint8_t (*s)[IW], int sr, int sc, int &dx, int &dy) {
    const int a00 = s[sr - 1][sc - 1], a01 = s[sr - 1][sc], a02 = s[sr - 1][sc + 1];
    const int a10 = s[sr][sc - 1], a12 = s[sr][sc + 1];
    const int a20 = s[sr + 1][sc - 1], a21 = s[sr + 1][sc], a22 = s[sr + 1][sc + 1];
    dx = 3 * (a02 - a00) + 10 * (a12 - a10) + 3 * (a22 - a20);
    dy = 3 * (a20 - a00) + 10 * (a21 - a01) + 3 * (a22 - a02);
}

// Stage rows [iy0, iy0 + IH) and columns [ix0, ix0 + IW) of an image.  The
// 16-byte path needs the source and its pitch 16-byte aligned (vec_ok).
template <int IH, int IW>
__device__ __forceinline__ void stage_tile(uint8_t (*s)[IW], const uint8_t *src, int w, int h, int pitch, int ix0,
                                           int iy0, bool vec_ok) {
    const bool interior = vec_ok && ix0 >= 0 && ix0 + IW <= w && iy0 >= 0 && iy0 + IH <= h;
    if (interior) {
        constexpr int C16 = IW / 16;
        for (int i = threadIdx.x; i < IH * C16; i += blockDim.x) {
            const int r = i / C16, c = i - r * C16;
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src + (size_t)(iy0 + r) * pitch + ix0) + c);
            *reinterpret_cast<uint4 *>(&s[r][c * 16]) = v;
        }
    } else {
        for (int i = threadIdx.x; i < IH * IW; i += blockDim.x) {
            const int r = i / IW, c = i - r * IW;
            const int sy = refl101(iy0 + r, h), sx = refl101(ix0 + c, w);
            s[r][c] = __ldg(src + (size_t)sy * pitch + sx);
        }
    }
}

// Copy the staged rows [r0, r0 + nr) x staged columns [c0, c0 + 128) to
// dst rows y0.. / columns x0.. (x0 a multiple of 128, dst rows 16-byte aligned).
template <int IW>
__device__ __forceinline__ void copy_out(const uint8_t (*s)[IW], int r0, int c0, int nr, uint8_t *dst, int dpitch,
                                         int x0, int y0, int w, int h) {
    for (int i = threadIdx.x; i < nr * 8; i += blockDim.x) {
        const int r = i >> 3, c = (i & 7) * 16;
        const int y = y0 + r, x = x0 + c;
        if (y >= h || x >= w) continue;
        uint8_t *d = dst + (size_t)y * dpitch + x;
        if (x + 16 <= w) {
            *reinterpret_cast<uint4 *>(d) = *reinterpret_cast<const uint4 *>(&s[r0 + r][c0 + c]);
        } else {
            for (int q = 0; q < 16 && x + q < w; ++q) d[q] = s[r0 + r][c0 + c + q];
        }
    }
}

// One output tile (tx, ty) of the pyramid step src -> dst; with GRAD also the
// Scharr planes of src over the matching 2*TW x 2*TH region, and with `copy`
// a copy of that src region (level 0 of a pyramid built from a caller image).
template <bool GRAD, int GT>
__device__ __forceinline__ void pyr_tile(const uint8_t *src, int w, int h, int spitch, bool vec_ok, uint8_t *dst,
                                         int dpitch, uint32_t *grad, int gpitch, uint8_t *copy, int cpitch, int tx,
                                         int ty, uint8_t (*s_in)[PD_IW], uint16_t (*s_v)[PD_VW]) {
    const int W = (w + 1) >> 1, H = (h + 1) >> 1;
    const int ox0 = tx * PD_TW, oy0 = ty * PD_TH;
    const int ix0 = 2 * ox0 - 16, iy0 = 2 * oy0 - 2;

    stage_tile<PD_IH, PD_IW>(s_in, src, w, h, spitch, ix0, iy0, vec_ok);
    __syncthreads();

    // vertical pass: s_v[r][c] for input column 2*ox0 - 2 + c (staged column c + 14)
    for (int i = threadIdx.x; i < PD_TH * PD_VW; i += blockDim.x) {
        const int r = i / PD_VW, c = i - r * PD_VW;
        const int cc = c + 14;
        s_v[r][c] = (uint16_t)(s_in[2 * r][cc] + 4 * s_in[2 * r + 1][cc] + 6 * s_in[2 * r + 2][cc] +
                               4 * s_in[2 * r + 3][cc] + s_in[2 * r + 4][cc]);
    }
    if (GRAD) {
        // gradients of the source level over [2*ox0, 2*ox0 + 2*TW) x [2*oy0, 2*oy0 + 2*TH)
        constexpr int GW = 2 * PD_TW, GH = 2 * PD_TH;
        for (int i = threadIdx.x; i < GH * (GW / 4); i += blockDim.x) {
            const int r = i / (GW / 4), x4 = (i - r * (GW / 4)) * 4;
            const int y = 2 * oy0 + r, x = 2 * ox0 + x4;
            if (y >= h || x >= w) continue;
            uint32_t g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int dx, dy;
                scharr_at<PD_IW>(s_in, r + 2, x4 + q + 16, dx, dy);
                g[q] = pack_grad<GT>(dx, dy);
            }
            uint32_t *d = grad + (size_t)y * gpitch + x;
            if (x + 3 < w) {
                *reinterpret_cast<uint4 *>(d) = make_uint4(g[0], g[1], g[2], g[3]);
            } else {
                for (int q = 0; q < 4 && x + q < w; ++q) d[q] = g[q];
            }
        }
    }
    if (copy) copy_out<PD_IW>(s_in, 2, 16, 2 * PD_TH, copy, cpitch, 2 * ox0, 2 * oy0, w, h);
    __syncthreads();
    // horizontal pass: 4 consecutive outputs per thread
    for (int i = threadIdx.x; i < PD_TH * (PD_TW / 4); i += blockDim.x) {
        const int r = i / (PD_TW / 4), x4 = (i - r * (PD_TW / 4)) * 4;
        const int oy = oy0 + r, ox = ox0 + x4;
        if (oy >= H || ox >= W) continue;
        const uint16_t *v = &s_v[r][2 * x4];
        uint32_t o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t s = v[2 * q] + 4u * v[2 * q + 1] + 6u * v[2 * q + 2] + 4u * v[2 * q + 3] + v[2 * q + 4];
            o[q] = (s + 128u) >> 8;
        }
        uint8_t *d = dst + (size_t)oy * dpitch + ox;
        if (ox + 3 < W) {
            *reinterpret_cast<uint32_t *>(d) = o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24);
        } else {
            for (int q = 0; q < 4 && ox + q < W; ++q) d[q] = (uint8_t)o[q];
        }
    }
}

// One Scharr tile (tx, ty) of a level; with `copy` also a copy of the tile.
template <int GT>
__device__ __forceinline__ void scharr_tile(const uint8_t *src, int w, int h, int spitch, bool vec_ok,
                                            uint32_t *grad, int gpitch, uint8_t *copy, int cpitch, int tx, int ty,
                                            uint8_t (*s_in)[SC_IW]) {
    const int x0 = tx * SC_TW, y0 = ty * SC_TH;
    stage_tile<SC_IH, SC_IW>(s_in, src, w, h, spitch, x0 - 16, y0 - 1, vec_ok);
    __syncthreads();
    for (int i = threadIdx.x; i < SC_TH * (SC_TW / 4); i += blockDim.x) {
        const int r = i / (SC_TW / 4), x4 = (i - r * (SC_TW / 4)) * 4;
        const int y = y0 + r, x = x0 + x4;
        if (y >= h || x >= w) continue;
        uint32_t g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int dx, dy;
            scharr_at<SC_IW>(s_in, r + 1, x4 + q + 16, dx, dy);
            g[q] = pack_grad<GT>(dx, dy);
        }
        uint32_t *d = grad + (size_t)y * gpitch + x;
        if (x + 3 < w) {
            *reinterpret_cast<uint4 *>(d) = make_uint4(g[0], g[1], g[2], g[3]);
        } else {
            for (int q = 0; q < 4 && x + q < w; ++q) d[q] = g[q];
        }
    }
    if (copy) {
        // SC_TW = 64 columns: copy with 16-byte stores per 16 columns
        for (int i = threadIdx.x; i < SC_TH * 4; i += blockDim.x) {
            const int r = i >> 2, c = (i & 3) * 16;
            const int y = y0 + r, x = x0 + c;
            if (y >= h || x >= w) continue;
            uint8_t *d = copy + (size_t)y * cpitch + x;
            if (x + 16 <= w) {
                *reinterpret_cast<uint4 *>(d) = *reinterpret_cast<const uint4 *>(&s_in[r + 1][c + 16]);
            } else {
                for (int q = 0; q < 16 && x + q < w; ++q) d[q] = s_in[r + 1][c + 16 + q];
            }
        }
    }
    __syncthreads();
}

template <bool GRAD, int GT>
__global__ void __launch_bounds__(PD_THREADS) k_pyrdown(const __grid_constant__ PyrJobs J) {
    __shared__ __align__(16) uint8_t s_in[PD_IH][PD_IW];
    __shared__ uint16_t s_v[PD_TH][PD_VW];
    int k = 0;
    while (k + 1 < J.njobs && (int)blockIdx.x >= J.j[k + 1].tile0) ++k;
    const PyrJob &jb = J.j[k];
    const int t = blockIdx.x - jb.tile0;
    const int ty = t / jb.tiles_x, tx = t - ty * jb.tiles_x;
    pyr_tile<GRAD, GT>(jb.src, jb.w, jb.h, jb.spitch, true, jb.dst, jb.dpitch, jb.grad, jb.gpitch, nullptr, 0, tx,
                       ty, s_in, s_v);
}

template <int GT>
__global__ void __launch_bounds__(SC_THREADS) k_scharr(const __grid_constant__ GradJobs J) {
    __shared__ __align__(16) uint8_t s_in[SC_IH][SC_IW];
    int k = 0;
    while (k + 1 < J.njobs && (int)blockIdx.x >= J.j[k + 1].tile0) ++k;
    const GradJob &jb = J.j[k];
    const int t = blockIdx.x - jb.tile0;
    const int ty = t / jb.tiles_x, tx = t - ty * jb.tiles_x;
    scharr_tile<GT>(jb.src, jb.w, jb.h, jb.spitch, true, jb.grad, jb.gpitch, nullptr, 0, tx, ty, s_in);
}

// --------------------------------------------------------- batched (persistent)
// Largest k with tile0[k] <= t over n jobs of stride `stride` ints.
__device__ __forceinline__ int find_job(const BLvlJob *jobs, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Launch `l` (< VT_MAX_LEVELS - 1): level l -> l+1 plus the Scharr planes of
// level l for every frame of the batch that has level l+1.  Level 0 reads the
// caller's image and writes the pyramid's level-0 copy from the same tile.
template <int GT>
__global__ void __launch_bounds__(PD_THREADS) k_pyr_batch(const uint8_t *tab, int l) {
    __shared__ __align__(16) uint8_t s_in[PD_IH][PD_IW];
    __shared__ uint16_t s_v[PD_TH][PD_VW];
    const BatchHdr *H = reinterpret_cast<const BatchHdr *>(tab);
    const int njobs = H->njobs[l], tiles = H->ntiles[l];
    const BFrame *frames = reinterpret_cast<const BFrame *>(tab + H->off_frames);
    const BLvlJob *jobs = reinterpret_cast<const BLvlJob *>(tab + H->off_jobs) + (size_t)l * H->cap_frames;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const BLvlJob jb = jobs[find_job(jobs, njobs, t)];
        const BFrame fr = frames[jb.frame];
        const Level src = fr.lv[l], dst = fr.lv[l + 1];
        const int tt = t - jb.tile0;
        const int ty = tt / jb.tiles_x, tx = tt - ty * jb.tiles_x;
        if (l == 0)
            pyr_tile<true, GT>(fr.img, src.w, src.h, fr.pitch, fr.vec_ok, dst.img, dst.pitch, src.grad, src.gpitch,
                               src.img, src.pitch, tx, ty, s_in, s_v);
        else
            pyr_tile<true, GT>(src.img, src.w, src.h, src.pitch, true, dst.img, dst.pitch, src.grad, src.gpitch,
                               nullptr, 0, tx, ty, s_in, s_v);
        __syncthreads();
    }
}

// Scharr planes of each frame's last level (which no pyramid step covers);
// a one-level pyramid also gets its level-0 copy here.
template <int GT>
__global__ void __launch_bounds__(SC_THREADS) k_scharr_batch(const uint8_t *tab) {
    __shared__ __align__(16) uint8_t s_in[SC_IH][SC_IW];
    const BatchHdr *H = reinterpret_cast<const BatchHdr *>(tab);
    const int njobs = H->njobs[VT_MAX_LEVELS - 1], tiles = H->ntiles[VT_MAX_LEVELS - 1];
    const BFrame *frames = reinterpret_cast<const BFrame *>(tab + H->off_frames);
    const BLvlJob *jobs =
        reinterpret_cast<const BLvlJob *>(tab + H->off_jobs) + (size_t)(VT_MAX_LEVELS - 1) * H->cap_frames;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const BLvlJob jb = jobs[find_job(jobs, njobs, t)];
        const BFrame fr = frames[jb.frame];
        const int l = fr.levels - 1;
        const Level lv = fr.lv[l];
        const int tt = t - jb.tile0;
        const int ty = tt / jb.tiles_x, tx = tt - ty * jb.tiles_x;
        if (l == 0)
            scharr_tile<GT>(fr.img, lv.w, lv.h, fr.pitch, fr.vec_ok, lv.grad, lv.gpitch, lv.img, lv.pitch, tx, ty,
                            s_in);
        else
            scharr_tile<GT>(lv.img, lv.w, lv.h, lv.pitch, true, lv.grad, lv.gpitch, nullptr, 0, tx, ty, s_in);
    }
}

int pyr_tiles(int w, int h, int &tiles_x) {
    const int W = (w + 1) / 2, H = (h + 1) / 2;
    tiles_x = (W + PD_TW - 1) / PD_TW;
    return tiles_x * ((H + PD_TH - 1) / PD_TH);
}

int scharr_tiles(int w, int h, int &tiles_x) {
    tiles_x = (w + SC_TW - 1) / SC_TW;
    return tiles_x * ((h + SC_TH - 1) / SC_TH);
}

vt_status launch_pyr_batch(const uint8_t *dev_tab, int maxL, int gtype, int grid_pyr, int grid_sc, cudaStream_t s) {
    for (int l = 0; l + 1 < maxL; ++l) {
        if (gtype == VT_GRAD_F16)
            k_pyr_batch<VT_GRAD_F16><<<grid_pyr, PD_THREADS, 0, s>>>(dev_tab, l);
        else
            k_pyr_batch<VT_GRAD_S16><<<grid_pyr, PD_THREADS, 0, s>>>(dev_tab, l);
    }
    if (gtype == VT_GRAD_F16)
        k_scharr_batch<VT_GRAD_F16><<<grid_sc, SC_THREADS, 0, s>>>(dev_tab);
    else
        k_scharr_batch<VT_GRAD_S16><<<grid_sc, SC_THREADS, 0, s>>>(dev_tab);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

int pyr_batch_blocks_per_sm() {
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pyr_batch<VT_GRAD_S16>, PD_THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_scharr_batch<VT_GRAD_S16>, SC_THREADS, 0);
    return a < b ? a : b;
}

void add_pyr_job(PyrJobs &jobs, int &blocks, const Level &src, const Level &dst, bool with_grad) {
    PyrJob &j = jobs.j[jobs.njobs++];
    j.src = src.img;
    j.dst = dst.img;
    j.grad = with_grad ? src.grad : nullptr;
    j.w = src.w;
    j.h = src.h;
    j.spitch = src.pitch;
    j.dpitch = dst.pitch;
    j.gpitch = src.gpitch;
    const int W = (src.w + 1) / 2, H = (src.h + 1) / 2;
    j.tiles_x = (W + PD_TW - 1) / PD_TW;
    const int tiles_y = (H + PD_TH - 1) / PD_TH;
    j.tile0 = blocks;
    blocks += j.tiles_x * tiles_y;
}

void add_grad_job(GradJobs &jobs, int &blocks, const Level &lv) {
    GradJob &j = jobs.j[jobs.njobs++];
    j.src = lv.img;
    j.grad = lv.grad;
    j.w = lv.w;
    j.h = lv.h;
    j.spitch = lv.pitch;
    j.gpitch = lv.gpitch;
    j.tiles_x = (lv.w + SC_TW - 1) / SC_TW;
    const int tiles_y = (lv.h + SC_TH - 1) / SC_TH;
    j.tile0 = blocks;
    blocks += j.tiles_x * tiles_y;
}

vt_status launch_pyrdown(const PyrJobs &jobs, int total_blocks, int gtype, cudaStream_t s) {
    if (jobs.njobs == 0 || total_blocks == 0) return VT_OK;
    const bool grad = jobs.j[0].grad != nullptr;
    if (!grad)
        k_pyrdown<false, VT_GRAD_S16><<<total_blocks, PD_THREADS, 0, s>>>(jobs);
    else if (gtype == VT_GRAD_F16)
        k_pyrdown<true, VT_GRAD_F16><<<total_blocks, PD_THREADS, 0, s>>>(jobs);
    else
        k_pyrdown<true, VT_GRAD_S16><<<total_blocks, PD_THREADS, 0, s>>>(jobs);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

vt_status launch_scharr(const GradJobs &jobs, int total_blocks, int gtype, cudaStream_t s) {
    if (jobs.njobs == 0 || total_blocks == 0) return VT_OK;
    if (gtype == VT_GRAD_F16)
        k_scharr<VT_GRAD_F16><<<total_blocks, SC_THREADS, 0, s>>>(jobs);
    else
        k_scharr<VT_GRAD_S16><<<total_blocks, SC_THREADS, 0, s>>>(jobs);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

// ------------------------------------------------------------------ host side
static vt_status alloc_pyramid(int w, int h, int levels, vt_pyramid **out) {
    vt_pyramid *p = (vt_pyramid *)calloc(1, sizeof(vt_pyramid));
    if (!p) return VT_ERR_OOM;
    p->w = w;
    p->h = h;
    p->levels = levels;
    p->gtype = VT_GRAD_NONE;
    cudaGetDevice(&p->device);
    size_t off = 256;  // the device copy of the level table sits at the start
    size_t img_off[VT_MAX_LEVELS], grad_off[VT_MAX_LEVELS];
    int lw = w, lh = h;
    for (int l = 0; l < levels; ++l) {
        Level &L = p->lv[l];
        L.w = lw;
        L.h = lh;
        L.pitch = round_up(lw, kImgPitchAlign);
        L.gpitch = round_up(lw, kGradPitchAlign);
        img_off[l] = off;
        off += ((size_t)L.pitch * lh + 255) / 256 * 256;
        lw = (lw + 1) / 2;
        lh = (lh + 1) / 2;
    }
    for (int l = 0; l < levels; ++l) {
        grad_off[l] = off;
        off += ((size_t)p->lv[l].gpitch * 4 * p->lv[l].h + 255) / 256 * 256;
    }
    off += 256;  // slack: wide loads of a footprint may read a few bytes past a row end
    if (cudaMalloc(&p->base, off) != cudaSuccess) {
        cudaGetLastError();
        free(p);
        return VT_ERR_OOM;
    }
    p->bytes = off;
    for (int l = 0; l < levels; ++l) {
        p->lv[l].img = (uint8_t *)p->base + img_off[l];
        p->lv[l].grad = (uint32_t *)((uint8_t *)p->base + grad_off[l]);
    }
    static_assert(sizeof(Level) * VT_MAX_LEVELS <= 256, "level table must fit its slot");
    p->dev_lv = (Level *)p->base;
    if (cudaMemcpy(p->dev_lv, p->lv, sizeof(Level) * VT_MAX_LEVELS, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p->base);
        free(p);
        return VT_ERR_CUDA;
    }
    *out = p;
    return VT_OK;
}

static vt_status check_build_args(const uint8_t *img, int w, int h, int pitch, int levels, vt_pyramid **out) {
    if (!img || !out || w <= 0 || h <= 0 || pitch < w || levels < 1 || levels > VT_MAX_LEVELS) return VT_ERR_ARG;
    // ceil-halving never reaches 0 px, so every level count up to VT_MAX_LEVELS is valid
    if (*out) {
        const vt_pyramid *p = *out;
        if (p->w != w || p->h != h || p->levels != levels) return VT_ERR_ARG;
    }
    return VT_OK;
}

static vt_status build_impl(const uint8_t *img, int w, int h, int pitch, int levels, int img_on_device, int gtype,
                            void *cuda_stream, vt_pyramid **out) {
    vt_status st = check_build_args(img, w, h, pitch, levels, out);
    if (st != VT_OK) return st;
    bool fresh = false;
    if (!*out) {
        st = alloc_pyramid(w, h, levels, out);
        if (st != VT_OK) return st;
        fresh = true;
    }
    vt_pyramid *p = *out;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const Level &L0 = p->lv[0];
    cudaError_t e = cudaMemcpy2DAsync(L0.img, L0.pitch, img, pitch, w, h,
                                      img_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (fresh) {
            vt_pyramid_free(p);
            *out = nullptr;
        }
        return VT_ERR_CUDA;
    }
    const bool grad = gtype != VT_GRAD_NONE;
    for (int l = 0; l + 1 < levels; ++l) {
        PyrJobs jobs;
        jobs.njobs = 0;
        int blocks = 0;
        add_pyr_job(jobs, blocks, p->lv[l], p->lv[l + 1], grad);
        st = launch_pyrdown(jobs, blocks, gtype, s);
        if (st != VT_OK) return st;
    }
    if (grad) {
        GradJobs gj;
        gj.njobs = 0;
        int blocks = 0;
        add_grad_job(gj, blocks, p->lv[levels - 1]);
        st = launch_scharr(gj, blocks, gtype, s);
        if (st != VT_OK) return st;
    }
    p->gtype = grad ? gtype : VT_GRAD_NONE;
    return VT_OK;
}

}  // namespace vt

using namespace vt;

extern "C" {

vt_status vt_pyramid_build(const uint8_t *img, int w, int h, int pitch, int levels, int img_on_device,
                           void *cuda_stream, vt_pyramid **out) {
    return build_impl(img, w, h, pitch, levels, img_on_device, VT_GRAD_NONE, cuda_stream, out);
}

vt_status vt_pyramid_build_grad(const uint8_t *img, int w, int h, int pitch, int levels, int img_on_device,
                                vt_grad_type t, void *cuda_stream, vt_pyramid **out) {
    if (t != VT_GRAD_S16 && t != VT_GRAD_F16) return VT_ERR_ARG;
    return build_impl(img, w, h, pitch, levels, img_on_device, (int)t, cuda_stream, out);
}

vt_status vt_gradients(vt_pyramid *p, vt_grad_type t, void *cuda_stream) {
    if (!p || (t != VT_GRAD_S16 && t != VT_GRAD_F16)) return VT_ERR_ARG;
    GradJobs gj;
    gj.njobs = 0;
    int blocks = 0;
    for (int l = 0; l < p->levels; ++l) add_grad_job(gj, blocks, p->lv[l]);
    vt_status st = launch_scharr(gj, blocks, (int)t, (cudaStream_t)cuda_stream);
    if (st == VT_OK) p->gtype = (int)t;
    return st;
}

vt_status vt_pyramid_create(int w, int h, int levels, vt_pyramid **out) {
    if (!out || w <= 0 || h <= 0 || levels < 1 || levels > VT_MAX_LEVELS) return VT_ERR_ARG;
    *out = nullptr;
    return alloc_pyramid(w, h, levels, out);
}

vt_status vt_pyramid_level(const vt_pyramid *p, int lvl, const uint8_t **ptr, int *w, int *h, int *pitch) {
    if (!p || lvl < 0 || lvl >= p->levels) return VT_ERR_ARG;
    if (ptr) *ptr = p->lv[lvl].img;
    if (w) *w = p->lv[lvl].w;
    if (h) *h = p->lv[lvl].h;
    if (pitch) *pitch = p->lv[lvl].pitch;
    return VT_OK;
}

vt_status vt_pyramid_grad(const vt_pyramid *p, int lvl, const void **ptr, int *pitch_pairs, vt_grad_type *t) {
    if (!p || lvl < 0 || lvl >= p->levels) return VT_ERR_ARG;
    if (ptr) *ptr = p->lv[lvl].grad;
    if (pitch_pairs) *pitch_pairs = p->lv[lvl].gpitch;
    if (t) *t = (vt_grad_type)p->gtype;
    return VT_OK;
}

vt_status vt_pyramid_info(const vt_pyramid *p, int *w, int *h, int *levels, size_t *device_bytes) {
    if (!p) return VT_ERR_ARG;
    if (w) *w = p->w;
    if (h) *h = p->h;
    if (levels) *levels = p->levels;
    if (device_bytes) *device_bytes = p->bytes;
    return VT_OK;
}

void vt_pyramid_free(vt_pyramid *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    cudaFree(p->base);
    free(p);
}

const char *vt_status_str(vt_status s) {
    switch (s) {
        case VT_OK: return "VT_OK";
        case VT_ERR_ARG: return "VT_ERR_ARG: invalid argument";
        case VT_ERR_OOM: return "VT_ERR_OOM: out of device memory";
        case VT_ERR_CUDA: return "VT_ERR_CUDA: CUDA call or launch failed";
        case VT_ERR_TIMEOUT: return "VT_ERR_TIMEOUT: a bounded wait ran out";
        case VT_ERR_UNSUPPORTED: return "VT_ERR_UNSUPPORTED: configuration not built";
    }
    return "unknown vt_status";
}

const char *vt_version(void) { return "vt 0.1 (sm_103a)"; }

}  // extern "C"
