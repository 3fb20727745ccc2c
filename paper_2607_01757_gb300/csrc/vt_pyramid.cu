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
constexpr int PD_VW = 2 * PD_TW + 8;   // vertical-pass columns (staged columns 12 .. 12 + PD_VW)
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

// Scharr (int16 output) of 4 consecutive columns x .. x+3 and 4 rows y0 ..
// y0+3 of the staged tile, two pixels per 32-bit operation.  A word holds two
// columns two apart in its 16-bit lanes: (x, x+2), (x+1, x+3), and the edge
// columns (x-1, x+4).  Per lane, the vertical smoothing V = 3 top + 10 mid +
// 3 bottom is at most 4080 and the biased difference D = bottom - top + 2048
// lies in [1793, 2303], so
//   dx + 32768 = V(x+1) - V(x-1) + 32768,
//   dy + 32768 = 3 D(x-1) + 10 D(x) + 3 D(x+1)      (bias 16 * 2048)
// both lie in [28688, 36848]: no lane ever borrows from or carries into its
// neighbour, and flipping bit 15 of a lane turns the biased value into the
// int16 two's complement of dx or dy.  Same results as the scalar form.
// `sr0` is the staged row above y0; `xr` the staged column offset of x.
__device__ __forceinline__ void scharr_4x4_s16(const uint8_t (*s)[PD_IW], int sr0, int xr, int x, int y0, int w,
                                               int h, uint32_t *grad, int gpitch) {
    uint32_t c13[3], c24[3], ce[3];  // rows above, centre, below
    auto load_row = [&](int sr, uint32_t &a13, uint32_t &a24, uint32_t &ae) {
        const uint32_t *wp = reinterpret_cast<const uint32_t *>(&s[sr][12 + xr]);
        const uint32_t a = wp[0], b = wp[1], c = wp[2];  // columns x-4 .. x+7
        a13 = b & 0x00FF00FFu;
        a24 = (b >> 8) & 0x00FF00FFu;
        ae = (a >> 24) | ((c << 16) & 0x00FF0000u);
    };
    load_row(sr0, c13[0], c24[0], ce[0]);
    load_row(sr0 + 1, c13[1], c24[1], ce[1]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        load_row(sr0 + 2 + i, c13[2], c24[2], ce[2]);
        const int y = y0 + i;
        if (y < h && x < w) {
            const uint32_t v13 = 3u * (c13[0] + c13[2]) + 10u * c13[1];
            const uint32_t v24 = 3u * (c24[0] + c24[2]) + 10u * c24[1];
            const uint32_t ve = 3u * (ce[0] + ce[2]) + 10u * ce[1];
            const uint32_t d13 = c13[2] + 0x08000800u - c13[0];
            const uint32_t d24 = c24[2] + 0x08000800u - c24[0];
            const uint32_t de = ce[2] + 0x08000800u - ce[0];
            const uint32_t vm = __byte_perm(ve, v24, 0x5410), vp = __byte_perm(v13, ve, 0x7632);  // (x-1, x+1), (x+2, x+4)
            const uint32_t dm = __byte_perm(de, d24, 0x5410), dp = __byte_perm(d13, de, 0x7632);
            const uint32_t dx13 = (v24 + 0x80008000u - vm) ^ 0x80008000u;  // columns (x, x+2)
            const uint32_t dx24 = (vp + 0x80008000u - v13) ^ 0x80008000u;  // columns (x+1, x+3)
            const uint32_t dy13 = (3u * (dm + d24) + 10u * d13) ^ 0x80008000u;
            const uint32_t dy24 = (3u * (d13 + dp) + 10u * d24) ^ 0x80008000u;
            const uint32_t g0 = __byte_perm(dx13, dy13, 0x5410), g2 = __byte_perm(dx13, dy13, 0x7632);
            const uint32_t g1 = __byte_perm(dx24, dy24, 0x5410), g3 = __byte_perm(dx24, dy24, 0x7632);
            uint32_t *d = grad + (size_t)y * gpitch + x;
            if (x + 3 < w) {
                *reinterpret_cast<uint4 *>(d) = make_uint4(g0, g1, g2, g3);
            } else {
                const uint32_t gq[4] = {g0, g1, g2, g3};
                for (int q = 0; q < 4 && x + q < w; ++q) d[q] = gq[q];
            }
        }
        c13[0] = c13[1], c24[0] = c24[1], ce[0] = ce[1];
        c13[1] = c13[2], c24[1] = c24[2], ce[1] = ce[2];
    }
}

// One output tile (tx, ty) of the pyramid step src -> dst; with GRAD also the
// Scharr planes of src over the matching 2*TW x 2*TH region, and with `copy`
// a copy of that src region (level 0 of a pyramid built from a caller image).
// Needs blockDim.x == PD_THREADS.
//
// The staged tile holds image columns ix0 .. ix0 + PD_IW with ix0 = 2*ox0 - 16
// and rows iy0 .. iy0 + PD_IH with iy0 = 2*oy0 - 2.
//  * vertical [1 4 6 4 1] pass on 32-bit words: the even and odd bytes of a
//    word are summed as two packed 16-bit lanes (at most 16 * 255 = 4080, no
//    carry between lanes), 4 columns per operation;
//  * horizontal pass: 4 outputs per thread from 6 packed column pairs, two
//    outputs per 32-bit operation;
//  * Scharr: each thread owns 4 columns x 4 rows and slides a 3-row window of
//    6 bytes per row (3 aligned word loads per row), with the separable form
//    dx = s(x+1) - s(x-1), s = 3 top + 10 mid + 3 bottom, and
//    dy = 3 d(x-1) + 10 d(x) + 3 d(x+1), d = bottom - top; int16 planes two
//    pixels per 32-bit operation (scharr_4x4_s16), half planes per pixel.
template <bool GRAD, int GT>
__device__ __forceinline__ void pyr_tile_compute(int w, int h, uint8_t *dst, int dpitch, uint32_t *grad, int gpitch,
                                                 uint8_t *copy, int cpitch, int tx, int ty,
                                                 uint8_t (*s_in)[PD_IW], uint16_t (*s_v)[PD_VW]);

template <bool GRAD, int GT>
__device__ __forceinline__ void pyr_tile(const uint8_t *src, int w, int h, int spitch, bool vec_ok, uint8_t *dst,
                                         int dpitch, uint32_t *grad, int gpitch, uint8_t *copy, int cpitch, int tx,
                                         int ty, uint8_t (*s_in)[PD_IW], uint16_t (*s_v)[PD_VW]) {
    stage_tile<PD_IH, PD_IW>(s_in, src, w, h, spitch, 2 * tx * PD_TW - 16, 2 * ty * PD_TH - 2, vec_ok);
    __syncthreads();
    pyr_tile_compute<GRAD, GT>(w, h, dst, dpitch, grad, gpitch, copy, cpitch, tx, ty, s_in, s_v);
}

// The computing part of pyr_tile on an already staged tile.
template <bool GRAD, int GT>
__device__ __forceinline__ void pyr_tile_compute(int w, int h, uint8_t *dst, int dpitch, uint32_t *grad, int gpitch,
                                                 uint8_t *copy, int cpitch, int tx, int ty,
                                                 uint8_t (*s_in)[PD_IW], uint16_t (*s_v)[PD_VW]) {
    const int W = (w + 1) >> 1, H = (h + 1) >> 1;
    const int ox0 = tx * PD_TW, oy0 = ty * PD_TH;

    // vertical pass: s_v[r][c] = sum_k [1 4 6 4 1]_k staged(2r + k, 12 + c)
    for (int i = threadIdx.x; i < PD_TH * (PD_VW / 4); i += PD_THREADS) {
        const int r = i / (PD_VW / 4), j = i - r * (PD_VW / 4);
        uint32_t lo[5], hi[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const uint32_t v = *reinterpret_cast<const uint32_t *>(&s_in[2 * r + k][12 + 4 * j]);
            lo[k] = v & 0x00FF00FFu;
            hi[k] = (v >> 8) & 0x00FF00FFu;
        }
        const uint32_t sl = lo[0] + lo[4] + 4u * (lo[1] + lo[3]) + 6u * lo[2];
        const uint32_t sh = hi[0] + hi[4] + 4u * (hi[1] + hi[3]) + 6u * hi[2];
        uint32_t *out = reinterpret_cast<uint32_t *>(&s_v[r][0]) + 2 * j;
        *reinterpret_cast<uint2 *>(out) = make_uint2(__byte_perm(sl, sh, 0x5410), __byte_perm(sl, sh, 0x7632));
    }
    if constexpr (GRAD && GT == VT_GRAD_S16) {
        const int g = threadIdx.x & 31, rg = threadIdx.x >> 5;
        scharr_4x4_s16(s_in, 4 * rg + 1, 4 * g, 2 * ox0 + 4 * g, 2 * oy0 + 4 * rg, w, h, grad, gpitch);
    } else if constexpr (GRAD) {
        const int g = threadIdx.x & 31, rg = threadIdx.x >> 5;
        const int xr = 4 * g, x = 2 * ox0 + xr;
        int t0[6], t1[6], t2[6];
        auto load_row = [&](int sr, int (&v)[6]) {
            const uint32_t *wp = reinterpret_cast<const uint32_t *>(&s_in[sr][12 + xr]);
            const uint32_t a = wp[0], b = wp[1], c = wp[2];
            v[0] = (int)(a >> 24);
            v[1] = (int)(b & 0xffu);
            v[2] = (int)((b >> 8) & 0xffu);
            v[3] = (int)((b >> 16) & 0xffu);
            v[4] = (int)(b >> 24);
            v[5] = (int)(c & 0xffu);
        };
        load_row(4 * rg + 1, t0);
        load_row(4 * rg + 2, t1);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            load_row(4 * rg + 3 + i, t2);
            const int y = 2 * oy0 + 4 * rg + i;
            if (y < h && x < w) {
                int sm[6], dd[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    sm[k] = 3 * (t0[k] + t2[k]) + 10 * t1[k];
                    dd[k] = t2[k] - t0[k];
                }
                uint32_t gq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    gq[q] = pack_grad<GT>(sm[q + 2] - sm[q], 3 * (dd[q] + dd[q + 2]) + 10 * dd[q + 1]);
                uint32_t *d = grad + (size_t)y * gpitch + x;
                if (x + 3 < w) {
                    *reinterpret_cast<uint4 *>(d) = make_uint4(gq[0], gq[1], gq[2], gq[3]);
                } else {
                    for (int q = 0; q < 4 && x + q < w; ++q) d[q] = gq[q];
                }
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                t0[k] = t1[k];
                t1[k] = t2[k];
            }
        }
    }
    if (copy) copy_out<PD_IW>(s_in, 2, 16, 2 * PD_TH, copy, cpitch, 2 * ox0, 2 * oy0, w, h);
    __syncthreads();
    // horizontal pass: 4 consecutive outputs per thread; output x uses
    // s_v columns 2x + 2 .. 2x + 6
    {
        const int r = threadIdx.x >> 4, x4 = (threadIdx.x & 15) * 4;
        const int oy = oy0 + r, ox = ox0 + x4;
        if (oy < H && ox < W) {
            // two outputs per 32-bit operation: lanes (o0, o1) and (o2, o3);
            // word k of the row holds s_v columns (2k, 2k+1) after the
            // offset, and output q needs columns 2q .. 2q+4, so lane pairs
            // (c, c+2) are gathered by byte permutes; a lane's sum is at
            // most 16 * 4080 = 65280 and never carries into its neighbour
            const uint32_t *pr = reinterpret_cast<const uint32_t *>(&s_v[r][0]) + x4 + 1;
            uint32_t p[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) p[k] = pr[k];
            auto lo2 = [](uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x5410); };
            auto hi2 = [](uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x7632); };
            auto down2 = [](uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t w4) {
                const uint32_t sum = w0 + w4 + 0x00800080u + 4u * (w1 + w3) + 6u * w2;
                return (sum >> 8) & 0x00FF00FFu;
            };
            const uint32_t w4 = lo2(p[2], p[3]);
            const uint32_t ra = down2(lo2(p[0], p[1]), hi2(p[0], p[1]), lo2(p[1], p[2]), hi2(p[1], p[2]), w4);
            const uint32_t rb = down2(w4, hi2(p[2], p[3]), lo2(p[3], p[4]), hi2(p[3], p[4]), lo2(p[4], p[5]));
            const uint32_t packed = __byte_perm(ra, rb, 0x6420);  // bytes o0, o1, o2, o3
            uint8_t *d = dst + (size_t)oy * dpitch + ox;
            if (ox + 3 < W) {
                *reinterpret_cast<uint32_t *>(d) = packed;
            } else {
                for (int q = 0; q < 4 && ox + q < W; ++q) d[q] = (uint8_t)(packed >> (8 * q));
            }
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
// level l for every frame of the batch whose tail starts above l (no Scharr
// planes for GT = VT_GRAD_NONE: the tracker computes gradients itself).  Level 0
// reads the caller's image and writes the pyramid's level-0 copy from the
// same tile (unless the frame is built in place).  The job list is first
// copied to shared memory so the per-tile job search does not chain global
// loads, and each job's source and destination are resolved on the host
// (BTileSrc), one load per tile, fetched a tile ahead.
constexpr int kJobsInSmem = 256;

// Six CTAs per SM (at most 40 registers a thread, no spills with the packed
// Scharr and horizontal passes): more tiles' loads in flight per SM.
template <int GT>
__global__ void __launch_bounds__(PD_THREADS, 6) k_pyr_batch(const uint8_t *tab, int l) {
    __shared__ __align__(16) uint8_t s_in[PD_IH][PD_IW];
    __shared__ uint16_t s_v[PD_TH][PD_VW];
    __shared__ BLvlJob s_jobs[kJobsInSmem];
    const BatchHdr *H = reinterpret_cast<const BatchHdr *>(tab);
    const int njobs = H->njobs[l], tiles = H->ntiles[l];
    if ((int)blockIdx.x >= tiles) return;
    const BLvlJob *gjobs = reinterpret_cast<const BLvlJob *>(tab + H->off_jobs) + (size_t)l * H->cap_frames;
    const bool in_smem = njobs <= kJobsInSmem;
    if (in_smem) {
        for (int i = threadIdx.x; i < njobs; i += blockDim.x) s_jobs[i] = gjobs[i];
        __syncthreads();
    }
    const BLvlJob *jobs = in_smem ? s_jobs : gjobs;
    const BTileSrc *tsrc = reinterpret_cast<const BTileSrc *>(tab + H->off_tsrc) + (size_t)l * H->cap_frames;
    // One thread resolves the CTA's next tile (its job's source record and
    // tile coordinates) into the other slot while the current tile is
    // computed, so no tile waits for the job search and the record's load.
    __shared__ BTileSrc s_ts[2];
    __shared__ int s_txy[2][2];
    auto locate = [&](int t, int k) {
        const int j = find_job(jobs, njobs, t);
        const int tt = t - jobs[j].tile0, nx = jobs[j].tiles_x;
        s_ts[k] = tsrc[j];
        s_txy[k][1] = tt / nx;
        s_txy[k][0] = tt - (tt / nx) * nx;
    };
    if (threadIdx.x == 0) locate(blockIdx.x, 0);  // the tables are complete before the first launch
    __syncthreads();
    pdl_wait();  // level l is the previous launch's output
    int k = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, k ^= 1) {
        if (t + (int)gridDim.x >= tiles) pdl_trigger();  // this CTA's last tile: the next launch may start
        const BTileSrc &ts = s_ts[k];  // fields read from shared memory where used
        const int tx = s_txy[k][0], ty = s_txy[k][1];
        // slot k ^ 1 was last read before the previous tile's closing barrier
        if (threadIdx.x == PD_THREADS - 32 && t + (int)gridDim.x < tiles) locate(t + (int)gridDim.x, k ^ 1);
        pyr_tile<GT != VT_GRAD_NONE, GT>(ts.src, ts.w, ts.h, ts.spitch, ts.vec_ok != 0, ts.dst, ts.dpitch, ts.grad,
                                         ts.gpitch, ts.copy, ts.cpitch, tx, ty, s_in, s_v);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ tail
constexpr int TAIL_THREADS = 1024;
constexpr int TAIL_A = kTailMaxPx;             // level c (<= kTailMaxPx pixels)
constexpr int TAIL_B = kTailMaxPx / 2 + 512;   // level c+1 (<= (w h + w + h + 1) / 4 pixels)
constexpr int TAIL_SMEM = TAIL_A + TAIL_B;

// First level the tail kernel builds: the first whose rows (at the
// pyramid's pitch) fit in kTailMaxPx bytes, or the last.
int tail_start_level(const vt_pyramid *p) {
    for (int l = 0; l < p->levels; ++l)
        if ((long)p->lv[l].pitch * p->lv[l].h <= kTailMaxPx) return l;
    return p->levels - 1;
}

// Row bands (CTAs) of a frame's tail: about 4096 pixels of level c each, at most 8.
int tail_parts(const vt_pyramid *p) {
    const int c = tail_start_level(p);
    const long px = (long)p->lv[c].w * p->lv[c].h;
    if ((long)p->lv[c].pitch * p->lv[c].h > kTailMaxPx) return 1;
    int n = (int)((px + 4095) / 4096);
    n = n < 1 ? 1 : (n > 8 ? 8 : n);
    return n < p->lv[c].h ? n : (p->lv[c].h > 0 ? p->lv[c].h : 1);
}

// Reflect-101 neighbours one step away (valid for any n >= 1).
__device__ __forceinline__ int refl_m1(int i, int n) { return i > 0 ? i - 1 : (n > 1 ? 1 : 0); }
__device__ __forceinline__ int refl_p1(int i, int n) { return i < n - 1 ? i + 1 : (n > 1 ? n - 2 : 0); }

// Scharr of rows [y0, y1) of a w x h level held in shared memory; warps take
// rows, lanes take columns.
template <int GT>
__device__ __forceinline__ void tail_scharr(const uint8_t *s, int stride, int w, int h, int y0, int y1,
                                            uint32_t *grad, int gpitch) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int y = y0 + (threadIdx.x >> 5); y < y1; y += nw) {
        const uint8_t *rm = s + refl_m1(y, h) * stride, *r0 = s + y * stride, *rp = s + refl_p1(y, h) * stride;
        uint32_t *g = grad + (size_t)y * gpitch;
        for (int x = lane; x < w; x += 32) {
            const int xm = refl_m1(x, w), xp = refl_p1(x, w);
            const int a00 = rm[xm], a01 = rm[x], a02 = rm[xp];
            const int a10 = r0[xm], a12 = r0[xp];
            const int a20 = rp[xm], a21 = rp[x], a22 = rp[xp];
            const int sm = 3 * (a02 - a00) + 10 * (a12 - a10) + 3 * (a22 - a20);
            const int dy = 3 * (a20 - a00) + 10 * (a21 - a01) + 3 * (a22 - a02);
            g[x] = pack_grad<GT>(sm, dy);
        }
    }
}

// pyrDown of a w x h level in shared memory (row stride `stride`) into d
// (shared, tight rows) and g (global).
__device__ __forceinline__ void tail_pyrdown(const uint8_t *s, int stride, int w, int h, uint8_t *d, uint8_t *g,
                                             int gpitch) {
    const int W = (w + 1) >> 1, H = (h + 1) >> 1;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int Y = threadIdx.x >> 5; Y < H; Y += nw) {
        const uint8_t *rows[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) rows[k] = s + refl101(2 * Y + k - 2, h) * stride;
        for (int X = lane; X < W; X += 32) {
            int cols[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) cols[k] = refl101(2 * X + k - 2, w);
            uint32_t acc = 0;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const uint8_t *r = rows[j];
                const uint32_t v = r[cols[0]] + r[cols[4]] + 4u * (r[cols[1]] + r[cols[3]]) + 6u * r[cols[2]];
                acc += (j == 2 ? 6u : (j == 1 || j == 3 ? 4u : 1u)) * v;
            }
            const uint8_t o = (uint8_t)((acc + 128u) >> 8);
            d[Y * W + X] = o;
            g[(size_t)Y * gpitch + X] = o;
        }
    }
}

// The tail of each frame's pyramid: the levels from c (the first level of at
// most kTailMaxPx pixels) down to the last, with their Scharr planes, from
// level c held in shared memory.  A frame's tail is split in `parts` row
// bands of level c's gradients, one CTA each; part 0 also builds the levels
// below c.  Level c comes from the tiled launches, or for c = 0 from the
// caller's image (part 0 then writes the level-0 copy).  A last level too
// large for shared memory (a large one-level pyramid) gets its Scharr planes
// tile by tile from global memory.
template <int GT>
__global__ void __launch_bounds__(TAIL_THREADS) k_pyr_tail(const uint8_t *tab) {
    extern __shared__ __align__(16) uint8_t tail_smem[];
    const BatchHdr *H = reinterpret_cast<const BatchHdr *>(tab);
    const int njobs = H->njobs[VT_MAX_LEVELS - 1];
    const BFrame *frames = reinterpret_cast<const BFrame *>(tab + H->off_frames);
    const BLvlJob *jobs =
        reinterpret_cast<const BLvlJob *>(tab + H->off_jobs) + (size_t)(VT_MAX_LEVELS - 1) * H->cap_frames;
    pdl_wait();  // level c is the previous launch's output
    for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
        if (j + (int)gridDim.x >= njobs) pdl_trigger();  // this CTA's last job
        const BLvlJob jb = jobs[j];
        const BFrame fr = frames[jb.frame];
        const int c = jb.aux;
        const int part = jb.tiles_x, parts = jb.tile0;  // tail lists: band index and band count
        const Level Lc = fr.lv[c];
        const uint8_t *src = c == 0 ? fr.img : Lc.img;
        const int sp = c == 0 ? fr.pitch : Lc.pitch;
        if ((long)Lc.pitch * Lc.h <= kTailMaxPx) {
            // level c in shared memory with the pyramid's row pitch
            uint8_t *cur = tail_smem, *nxt = tail_smem + TAIL_A;
            if (c > 0) {  // a pyramid level: 16-byte aligned rows
                const int n16 = Lc.pitch * Lc.h / 16;
                const uint4 *g4 = reinterpret_cast<const uint4 *>(Lc.img);
                uint4 *s4 = reinterpret_cast<uint4 *>(cur);
                for (int i = threadIdx.x; i < n16; i += blockDim.x) s4[i] = __ldg(g4 + i);
            } else {  // the caller's image: any alignment
                const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
                for (int y = threadIdx.x >> 5; y < Lc.h; y += nw) {
                    const uint8_t *sr = src + (size_t)y * sp;
                    for (int x = lane; x < Lc.w; x += 32) {
                        const uint8_t v = sr[x];
                        cur[y * Lc.pitch + x] = v;
                        if (part == 0 && src != Lc.img) Lc.img[(size_t)y * Lc.pitch + x] = v;
                    }
                }
            }
            __syncthreads();
            const int band = (Lc.h + parts - 1) / parts;
            const int y0 = part * band, y1 = min(Lc.h, y0 + band);
            if constexpr (GT != VT_GRAD_NONE) tail_scharr<GT>(cur, Lc.pitch, Lc.w, Lc.h, y0, y1, Lc.grad, Lc.gpitch);
            if (part == 0) {
                int stride = Lc.pitch;
                for (int l = c; l + 1 < fr.levels; ++l) {
                    const Level L = fr.lv[l], N = fr.lv[l + 1];
                    tail_pyrdown(cur, stride, L.w, L.h, nxt, N.img, N.pitch);
                    __syncthreads();
                    if constexpr (GT != VT_GRAD_NONE) tail_scharr<GT>(nxt, N.w, N.w, N.h, 0, N.h, N.grad, N.gpitch);
                    uint8_t *t = cur;
                    cur = nxt;
                    nxt = t;
                    stride = N.w;
                }
            }
        } else if (part == 0) {
            if constexpr (GT != VT_GRAD_NONE) {
                uint8_t (*s_in)[SC_IW] = reinterpret_cast<uint8_t (*)[SC_IW]>(tail_smem);
                int tiles_x;
                const int tiles = scharr_tiles(Lc.w, Lc.h, tiles_x);
                for (int t = 0; t < tiles; ++t) {
                    const int ty = t / tiles_x, tx = t - ty * tiles_x;
                    scharr_tile<GT>(src, Lc.w, Lc.h, sp, c == 0 ? fr.vec_ok != 0 : true, Lc.grad, Lc.gpitch,
                                    (c == 0 && src != Lc.img) ? Lc.img : nullptr, Lc.pitch, tx, ty, s_in);
                }
            } else if (c == 0 && src != Lc.img) {  // no gradients: only the level-0 copy of a large one-level pyramid
                const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
                for (int y = threadIdx.x >> 5; y < Lc.h; y += nw)
                    for (int x = lane; x < Lc.w; x += 32) Lc.img[(size_t)y * Lc.pitch + x] = src[(size_t)y * sp + x];
            }
        }
        __syncthreads();
    }
}

int pyr_tiles(int w, int h, int &tiles_x) {
    const int W = (w + 1) / 2, H = (h + 1) / 2;
    tiles_x = (W + PD_TW - 1) / PD_TW;
    return tiles_x * ((H + PD_TH - 1) / PD_TH);
}

__host__ __device__ int scharr_tiles(int w, int h, int &tiles_x) {
    tiles_x = (w + SC_TW - 1) / SC_TW;
    return tiles_x * ((h + SC_TH - 1) / SC_TH);
}

vt_status launch_pyr_batch(const uint8_t *dev_tab, int tiled_launches, int gtype, int grid_pyr, int grid_tail,
                           cudaStream_t s, cudaEvent_t *ev) {
    static const bool attr = [] {  // once, thread-safe static initialisation
        return cudaFuncSetAttribute(k_pyr_tail<VT_GRAD_S16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TAIL_SMEM) == cudaSuccess &&
               cudaFuncSetAttribute(k_pyr_tail<VT_GRAD_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TAIL_SMEM) == cudaSuccess &&
               cudaFuncSetAttribute(k_pyr_tail<VT_GRAD_NONE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TAIL_SMEM) == cudaSuccess;
    }();
    (void)attr;
    // every launch after the first overlaps its start with the previous one's
    // end (programmatic dependent launch), except where an event is recorded
    // in between for per-launch timing
    auto pyr = gtype == VT_GRAD_F16 ? k_pyr_batch<VT_GRAD_F16>
                                    : (gtype == VT_GRAD_NONE ? k_pyr_batch<VT_GRAD_NONE> : k_pyr_batch<VT_GRAD_S16>);
    auto tail = gtype == VT_GRAD_F16 ? k_pyr_tail<VT_GRAD_F16>
                                     : (gtype == VT_GRAD_NONE ? k_pyr_tail<VT_GRAD_NONE> : k_pyr_tail<VT_GRAD_S16>);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < tiled_launches && e == cudaSuccess; ++l) {
        e = launch_pdl(pyr, grid_pyr, PD_THREADS, 0, s, l > 0 && !ev, dev_tab, l);
        if (ev && ev[l]) cudaEventRecord(ev[l], s);
    }
    if (e == cudaSuccess) e = launch_pdl(tail, grid_tail, TAIL_THREADS, TAIL_SMEM, s, tiled_launches > 0 && !ev, dev_tab);
    if (ev && ev[tiled_launches]) cudaEventRecord(ev[tiled_launches], s);
    return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

int pyr_batch_blocks_per_sm() {
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pyr_batch<VT_GRAD_S16>, PD_THREADS, 0);
    return a;
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
// `level0` (nullable): the caller's level-0 buffer (row pitch `pitch0`); the
// allocation then holds only the levels above 0 and the planes.
static vt_status alloc_pyramid(int w, int h, int levels, vt_pyramid **out, uint8_t *level0 = nullptr,
                               int pitch0 = 0) {
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
        L.pitch = (l == 0 && level0) ? pitch0 : round_up(lw, kImgPitchAlign);
        L.gpitch = round_up(lw, kGradPitchAlign);
        img_off[l] = off;
        if (l > 0 || !level0) off += ((size_t)L.pitch * lh + 255) / 256 * 256;
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
        p->lv[l].img = (l == 0 && level0) ? level0 : (uint8_t *)p->base + img_off[l];
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
    if (img == L0.img && pitch != L0.pitch) return VT_ERR_ARG;
    // a frame already in level 0 (vt_pyramid_upload) is built in place
    cudaError_t e = img == L0.img ? cudaSuccess
                                  : cudaMemcpy2DAsync(L0.img, L0.pitch, img, pitch, w, h,
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

vt_status vt_pyramid_upload(vt_pyramid *p, const uint8_t *img, int pitch, int img_on_device, void *cuda_stream) {
    if (!p || !img || pitch < p->w) return VT_ERR_ARG;
    const Level &L0 = p->lv[0];
    if (cudaMemcpy2DAsync(L0.img, L0.pitch, img, pitch, p->w, p->h,
                          img_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          (cudaStream_t)cuda_stream) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    return VT_OK;
}

vt_status vt_pyramid_create(int w, int h, int levels, vt_pyramid **out) {
    if (!out || w <= 0 || h <= 0 || levels < 1 || levels > VT_MAX_LEVELS) return VT_ERR_ARG;
    *out = nullptr;
    return alloc_pyramid(w, h, levels, out);
}

vt_status vt_pyramid_create_on(const uint8_t *level0, int pitch, size_t level0_bytes, int w, int h, int levels,
                               vt_pyramid **out) {
    if (!out || !level0 || w <= 0 || h <= 0 || levels < 1 || levels > VT_MAX_LEVELS) return VT_ERR_ARG;
    if ((uintptr_t)level0 % 16 != 0 || pitch % 16 != 0 || pitch < w) return VT_ERR_ARG;
    if (level0_bytes < (size_t)pitch * h + 32) return VT_ERR_ARG;
    *out = nullptr;
    return alloc_pyramid(w, h, levels, out, const_cast<uint8_t *>(level0), pitch);
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
