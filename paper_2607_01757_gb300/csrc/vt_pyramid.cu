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

// Stage rows [iy0, iy0 + IH) and columns [ix0, ix0 + IW) of an image.
template <int IH, int IW>
__device__ __forceinline__ void stage_tile(uint8_t (*s)[IW], const uint8_t *src, int w, int h, int pitch, int ix0,
                                           int iy0, int nthreads) {
    const bool interior = ix0 >= 0 && ix0 + IW <= w && iy0 >= 0 && iy0 + IH <= h;
    if (interior) {
        constexpr int C16 = IW / 16;
        for (int i = threadIdx.x; i < IH * C16; i += nthreads) {
            const int r = i / C16, c = i - r * C16;
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src + (size_t)(iy0 + r) * pitch + ix0) + c);
            *reinterpret_cast<uint4 *>(&s[r][c * 16]) = v;
        }
    } else {
        for (int i = threadIdx.x; i < IH * IW; i += nthreads) {
            const int r = i / IW, c = i - r * IW;
            const int sy = refl101(iy0 + r, h), sx = refl101(ix0 + c, w);
            s[r][c] = __ldg(src + (size_t)sy * pitch + sx);
        }
    }
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
    const int W = (jb.w + 1) >> 1, H = (jb.h + 1) >> 1;
    const int ox0 = tx * PD_TW, oy0 = ty * PD_TH;
    const int ix0 = 2 * ox0 - 16, iy0 = 2 * oy0 - 2;

    stage_tile<PD_IH, PD_IW>(s_in, jb.src, jb.w, jb.h, jb.spitch, ix0, iy0, PD_THREADS);
    __syncthreads();

    // vertical pass: s_v[r][c] for input column 2*ox0 - 2 + c (staged column c + 14)
    for (int i = threadIdx.x; i < PD_TH * PD_VW; i += PD_THREADS) {
        const int r = i / PD_VW, c = i - r * PD_VW;
        const int cc = c + 14;
        s_v[r][c] = (uint16_t)(s_in[2 * r][cc] + 4 * s_in[2 * r + 1][cc] + 6 * s_in[2 * r + 2][cc] +
                               4 * s_in[2 * r + 3][cc] + s_in[2 * r + 4][cc]);
    }
    if (GRAD) {
        // gradients of the source level over [2*ox0, 2*ox0 + 2*TW) x [2*oy0, 2*oy0 + 2*TH)
        constexpr int GW = 2 * PD_TW, GH = 2 * PD_TH;
        for (int i = threadIdx.x; i < GH * (GW / 4); i += PD_THREADS) {
            const int r = i / (GW / 4), x4 = (i - r * (GW / 4)) * 4;
            const int y = 2 * oy0 + r, x = 2 * ox0 + x4;
            if (y >= jb.h || x >= jb.w) continue;
            uint32_t g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int dx, dy;
                scharr_at<PD_IW>(s_in, r + 2, x4 + q + 16, dx, dy);
                g[q] = pack_grad<GT>(dx, dy);
            }
            uint32_t *d = jb.grad + (size_t)y * jb.gpitch + x;
            if (x + 3 < jb.w) {
                *reinterpret_cast<uint4 *>(d) = make_uint4(g[0], g[1], g[2], g[3]);
            } else {
                for (int q = 0; q < 4 && x + q < jb.w; ++q) d[q] = g[q];
            }
        }
    }
    __syncthreads();
    // horizontal pass: 4 consecutive outputs per thread
    for (int i = threadIdx.x; i < PD_TH * (PD_TW / 4); i += PD_THREADS) {
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
        uint8_t *d = jb.dst + (size_t)oy * jb.dpitch + ox;
        if (ox + 3 < W) {
            *reinterpret_cast<uint32_t *>(d) = o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24);
        } else {
            for (int q = 0; q < 4 && ox + q < W; ++q) d[q] = (uint8_t)o[q];
        }
    }
}

template <int GT>
__global__ void __launch_bounds__(SC_THREADS) k_scharr(const __grid_constant__ GradJobs J) {
    __shared__ __align__(16) uint8_t s_in[SC_IH][SC_IW];
    int k = 0;
    while (k + 1 < J.njobs && (int)blockIdx.x >= J.j[k + 1].tile0) ++k;
    const GradJob &jb = J.j[k];
    const int t = blockIdx.x - jb.tile0;
    const int ty = t / jb.tiles_x, tx = t - ty * jb.tiles_x;
    const int x0 = tx * SC_TW, y0 = ty * SC_TH;
    stage_tile<SC_IH, SC_IW>(s_in, jb.src, jb.w, jb.h, jb.spitch, x0 - 16, y0 - 1, SC_THREADS);
    __syncthreads();
    for (int i = threadIdx.x; i < SC_TH * (SC_TW / 4); i += SC_THREADS) {
        const int r = i / (SC_TW / 4), x4 = (i - r * (SC_TW / 4)) * 4;
        const int y = y0 + r, x = x0 + x4;
        if (y >= jb.h || x >= jb.w) continue;
        uint32_t g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int dx, dy;
            scharr_at<SC_IW>(s_in, r + 1, x4 + q + 16, dx, dy);
            g[q] = pack_grad<GT>(dx, dy);
        }
        uint32_t *d = jb.grad + (size_t)y * jb.gpitch + x;
        if (x + 3 < jb.w) {
            *reinterpret_cast<uint4 *>(d) = make_uint4(g[0], g[1], g[2], g[3]);
        } else {
            for (int q = 0; q < 4 && x + q < jb.w; ++q) d[q] = g[q];
        }
    }
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
    size_t off = 0;
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
