// Warp-per-feature pyramidal Lucas-Kanade (K3), shared by the single-pair
// kernels (vt_klt.cu) and the batched persistent kernel (vt_batch.cu) so that
// a point gives bit-identical results alone or in a batch.
//
// The method (textbook coarse-to-fine LK, the tracker the paper uses in
// Sec. IV / Table I; cross-camera check of Sec. V-A):
//   per level l = L-1 .. 0, u_l = u / 2^l:
//     T(x), grad T(x): bilinear samples of I_l and its Scharr planes at u_l + x
//     G = sum grad T grad T^T, reject if lambda_min / (win^2 255^2) < min_eig
//     iterate: q = u_l + g_l + nu (bound test), r = T - J_l(q + x),
//              b = sum r grad T, eta = G^-1 b, nu += eta, stop |eta|^2 < eps^2
//     g_{l-1} = 2 (g_l + nu)
//   result v = u + g_0 + nu (bound test), error = mean |T - J_0(v + x)|.
//
// Mapping to the warp: the window is cut into short runs of rows of one
// column, a lane owning one or two runs (KRuns), so all 32 lanes work on the
// win^2 samples.  Every window sample of one Newton
// iteration shares the same fractional bilinear weights (bx, by), so
// b = sum (T - J(q + x)) grad T expands exactly into bx, by and eight moments
// of the integer footprint of J under the window (cell_moments).  A sweep
// over the footprint is needed only when the integer part of q changes;
// iterations that stay in the same cell reuse the moments.  The template and
// its gradients stay in registers (three floats per owned sample); the image and
// gradient window it is sampled from, and each footprint, are staged in
// per-warp shared memory by cp.async.  Sums over the window are per-lane FP32
// sums over rows followed by a warp reduction that leaves bit-identical
// totals in every lane (an XOR butterfly, or a reduce-scatter and broadcast),
// so control flow stays warp-uniform.
#pragma once

#include <climits>

#include "vt_internal.cuh"

namespace vt {

struct KPyr {
    Level lv[VT_MAX_LEVELS];
};

struct KOut {
    float x, y;     // level-0 result (last estimate when lost)
    float err;      // mean |T - J| (0 when lost)
    float lmin;     // normalised lambda_min at the last level examined
    int status;     // 1 tracked
    int reason;     // VT_TRACKED / VT_LOST_*
    int iters;      // Newton iterations over all levels (and both passes)
    int tmpl;       // template extractions (window sweeps of 27 FLOP per sample)
    int errp;       // error passes (window sweeps of 9 FLOP per sample)
    int sweeps;     // footprint sweeps the Newton iterations actually needed
};

// Algorithmic FLOPs of a tracked point: per window sample 27 for a template
// sweep (bilinear I, Ix, Iy: 3 x 7; G: 3 FMA), 12 for a Newton sweep
// (bilinear J: 7; residual: 1; b: 2 FMA) and 9 for the error sweep.
__device__ __forceinline__ int klt_flops(int win, const KOut &o) {
    return win * win * (27 * o.tmpl + 12 * o.iters + 9 * o.errp);
}

constexpr unsigned kFull = 0xffffffffu;

// Resident CTAs per SM the tracking kernels are register-budgeted for
// (4-warp CTAs): 4 for windows up to 21 (128 registers per thread).
template <int WIN>
struct KltOcc {
    static constexpr int min_blocks = WIN <= 21 ? 4 : 3;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
    return v;
}

// Warp totals of eight per-lane values, delivered to every lane: the three
// top butterfly levels are a reduce-scatter (each halves the set a lane
// carries), the last two reduce the lane's single value, and the eight totals
// are broadcast from lanes 0, 4, .., 28.  17 shuffles instead of 5 x 8.
__device__ __forceinline__ void warp_sum8(const float (&a)[8], int lane, float (&m)[8]) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float b[4], c[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = h16 ? a[k] : a[k + 4], keep = h16 ? a[k + 4] : a[k];
        b[k] = keep + __shfl_xor_sync(kFull, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = h8 ? b[k] : b[k + 2], keep = h8 ? b[k + 2] : b[k];
        c[k] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    const float send = h4 ? c[0] : c[1], keep = h4 ? c[1] : c[0];
    float d = keep + __shfl_xor_sync(kFull, send, 4);
    d += __shfl_xor_sync(kFull, d, 2);
    d += __shfl_xor_sync(kFull, d, 1);
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k] = __shfl_sync(kFull, d, 4 * k);  // lane 4k holds total k
}

// Warp totals of three per-lane values the same way (the set padded to four
// with a zero; totals broadcast from lanes 0, 8, 16): 9 shuffles instead of
// 5 x 3.
__device__ __forceinline__ void warp_sum3(float x, float y, float z, int lane, float &sx, float &sy, float &sz) {
    const bool h16 = lane & 16, h8 = lane & 8;
    const float s0 = h16 ? x : z, k0 = h16 ? z : x;
    const float s1 = h16 ? y : 0.f, k1 = h16 ? 0.f : y;
    const float b0 = k0 + __shfl_xor_sync(kFull, s0, 16);
    const float b1 = k1 + __shfl_xor_sync(kFull, s1, 16);
    const float sd = h8 ? b0 : b1, kd = h8 ? b1 : b0;
    float d = kd + __shfl_xor_sync(kFull, sd, 8);
    d += __shfl_xor_sync(kFull, d, 4);
    d += __shfl_xor_sync(kFull, d, 2);
    d += __shfl_xor_sync(kFull, d, 1);
    sx = __shfl_sync(kFull, d, 0);
    sy = __shfl_sync(kFull, d, 8);
    sz = __shfl_sync(kFull, d, 16);
}

// A byte as a float (exact; differences of two are exact integers).  The
// conversion runs on its own pipe, off the integer pipe that an OR-with-2^23
// conversion would load.
__device__ __forceinline__ float u8f(uint32_t v) { return __uint2float_rn(v); }

template <int GT>
__device__ __forceinline__ void unpack_grad(uint32_t v, float &gx, float &gy) {
    if (GT == VT_GRAD_S16) {
        gx = (float)(int)(int16_t)(v & 0xffffu);
        gy = (float)((int)v >> 16);
    } else {
        const __half2 h = *reinterpret_cast<const __half2 *>(&v);
        const float2 f = __half22float2(h);
        gx = f.x;
        gy = f.y;
    }
}

// Scale from the stored gradient unit to grey levels per pixel (gradients
// computed on the fly, VT_GRAD_NONE, are raw Scharr like VT_GRAD_S16).
template <int GT>
__device__ __forceinline__ constexpr float grad_unit() { return GT == VT_GRAD_F16 ? 1.0f : 0.03125f; }

// a b - c d by Kahan's FMA scheme: w = c d rounded, its rounding error
// c d - w is exact (one FMA), and the result is round(a b - w) minus that
// error.  Relative error at most 2 ulp and the sign exact (Jeannerod, Louvet
// & Muller, Math. Comp. 82, 2013) -- as good as FP64 products rounded to FP32,
// but on the FP32 pipes: this GPU's FP64 pipe retires about 2 lanes per clock
// per SM, and an FP64 determinant and divides per template kept it 42 % busy.
__device__ __forceinline__ float kdiff(float a, float b, float c, float d) {
    const float w = c * d;
    return fmaf(a, b, -w) - fmaf(c, d, -w);
}

// 2^-l exactly.
__device__ __forceinline__ float pow2neg(int l) { return __int_as_float((127 - l) << 23); }

// Per-warp shared scratch: the staged (win + 1)^2 window of a level image --
// the footprint of J for one sweep, or the template's source -- in win + 1
// rows of NC 16-byte chunks, and the template's gradient window in win + 1
// rows of NG 16-byte chunks.
template <int WIN>
struct KSmem {
    static constexpr int NC = (WIN + 31) / 16;  // 16-byte chunks per staged row: cover 15 + win + 1 bytes
    static constexpr int JS = NC * 16;          // staged row stride in bytes
    static_assert(JS >= 15 + WIN + 1 && JS - 1 - WIN <= 32, "a staged row covers the footprint row and reads "
                                                              "at most 32 bytes past it (the allocation keeps 256)");
    uint8_t j[(WIN + 1) * JS];
    static constexpr int NG = (4 * (3 + WIN + 1) + 15) / 16;  // 16-byte chunks per staged gradient row
    static constexpr int GS = NG * 4;                         // staged gradient row stride in words
    static_assert(GS >= 3 + WIN + 1 && 4 * (GS - WIN - 1) <= 32, "a staged gradient row covers the window row "
                                                                 "and reads at most 32 bytes past it");
    uint32_t g[(WIN + 1) * GS];
    uint8_t t[(WIN + 1) * JS];  // the template's image window, kept while footprints are staged (FP64 levels)
    // zeros that a lane's run outside the window reads instead of the staged
    // windows (its template samples and error terms are then exactly zero
    // without a select per sample): RL + 1 rows of two bytes / words at the
    // staged strides (RL = samples per run)
    static constexpr int RLZ = WIN / (WIN == 31 ? 1 : 3);
    uint8_t zj[RLZ * JS + 16];
    uint32_t zg[RLZ * GS + 4];
};

// Clear a warp's zero rows (once per kernel, before the first point).
template <int WIN>
__device__ __forceinline__ void ksmem_init(KSmem<WIN> &sm, int lane) {
    for (int k = lane; k < (int)sizeof(sm.zj); k += 32) sm.zj[k] = 0;
    for (int k = lane; k < (int)(sizeof(sm.zg) / 4); k += 32) sm.zg[k] = 0;
    __syncwarp();
}

// Which window samples a lane owns.  The win x win window is cut into runs
// of RL consecutive rows of one column (D bands of RL rows, win * D runs in
// all, numbered band by band so that lanes reading at the same time touch at
// most two staged rows: fewer shared-memory bank conflicts); lane l owns
// runs l, l + 32, ... (at most RPL).  A lane walks each of
// its runs down the column, reading footprint rows r0 .. r0 + RL and the
// neighbouring column from shared memory, so every lane works (with one
// column per lane, 32 - win lanes would idle) and the right neighbour needs
// no shuffle.  The per-sample arithmetic does not depend on the layout; only
// the grouping of the per-lane partial sums does.
template <int WIN>
struct KRuns {
    static constexpr int D = WIN == 31 ? 1 : 3;
    static_assert(WIN % D == 0, "runs tile a column");
    static constexpr int RL = WIN / D;          // samples per run
    static constexpr int NR = WIN * D;          // runs in the window
    static constexpr int RPL = (NR + 31) / 32;  // runs per lane
    static constexpr int NS = RPL * RL;         // samples a lane holds
};

// Run i of a lane: column c, first row r0, and whether it lies in the window
// (a lane's last run may not: it then reads run 0's addresses and its
// samples weigh zero).
template <int WIN>
__device__ __forceinline__ void run_of(int lane, int i, int &c, int &r0, bool &valid) {
    constexpr int RL = KRuns<WIN>::RL;
    const int k = lane + 32 * i;
    valid = k < KRuns<WIN>::NR;
    const int kk = valid ? k : 0;
    const int band = kk / WIN;
    c = kk - band * WIN;
    r0 = band * RL;
}

// Gradient window of a level without stored gradients (VT_GRAD_NONE): lane c
// (c <= win) computes the raw Scharr responses of staged column c -- the
// integers the pyramid kernels would have stored for the replicate-clamped
// pixel (reflect-101 neighbours) -- and stores them as int16 pairs in the
// staged gradient window, with the pixel itself in the staged image window,
// so the template is then sampled exactly as from stored int16 gradients.
//
// Per image row y the lane forms d(y) = I(y, x+1) - I(y, x-1) and
// s(y) = 3 I(y, x-1) + 10 I(y, x) + 3 I(y, x+1); the gradient of row y is
// dx = 3 d(y-1) + 10 d(y) + 3 d(y+1), dy = s(y+1) - s(y-1).  The clamped rows
// R(k) = clamp(y0 + k) are read once each (a rolling window): for an
// interior row R(r) its neighbours are R(r-1) and R(r+1); a row at the
// image's first or last line takes its reflected neighbour (row 1 or h-2)
// on both sides instead.
template <int WIN>
__device__ __forceinline__ void stage_window_otf(const Level &L, int x0, int y0, int lane, KSmem<WIN> &sm) {
    constexpr int JS = KSmem<WIN>::JS, GS = KSmem<WIN>::GS;
    const bool ld = lane <= WIN;
    const int q = clampi(x0 + lane, 0, L.w - 1);
    const int qm = refl101(q - 1, L.w), qp = refl101(q + 1, L.w);
    const int hm1 = L.h - 1;
    auto terms = [&](int y, int &d, int &sm_, int &c) {
        const uint8_t *rp = L.img + (size_t)y * L.pitch;
        int a = 0, b = 0, e = 0;
        if (ld) {
            a = __ldg(rp + qm);
            b = __ldg(rp + q);
            e = __ldg(rp + qp);
        }
        d = e - a;
        sm_ = 3 * (a + e) + 10 * b;
        c = b;
    };
    // reflected neighbours of the first and last image rows (used only when
    // the window reaches them)
    int dt = 0, st = 0, db = 0, sb = 0, unused;
    if (y0 <= 0 || hm1 == 0) terms(refl101(-1, L.h), dt, st, unused);
    if (y0 + WIN >= hm1) terms(refl101(L.h, L.h), db, sb, unused);
    int dm, sm_m, cm, d0, s0, c0;
    terms(clampi(y0 - 1, 0, hm1), dm, sm_m, cm);
    terms(clampi(y0, 0, hm1), d0, s0, c0);
    __syncwarp();
#pragma unroll
    for (int r = 0; r <= WIN; ++r) {
        const int yc = clampi(y0 + r, 0, hm1);
        int dp, sp, cp;
        terms(clampi(y0 + r + 1, 0, hm1), dp, sp, cp);
        const bool top = yc == 0, bot = yc == hm1;
        const int du = top ? dt : (bot ? db : dm), su = top ? st : (bot ? sb : sm_m);
        const int dd = top ? dt : (bot ? db : dp), sd = top ? st : (bot ? sb : sp);
        const int gx = 3 * (du + dd) + 10 * d0, gy = sd - su;
        if (ld) {
            sm.j[r * JS + lane] = (uint8_t)c0;
            sm.g[r * GS + lane] = (uint32_t)(uint16_t)(int16_t)gx | ((uint32_t)(uint16_t)(int16_t)gy << 16);
        }
        dm = d0;
        sm_m = s0;
        d0 = dp;
        s0 = sp;
        c0 = cp;
    }
    __syncwarp();
}

// Sample the template of level `L` around (ux, uy) at the lane's window
// samples (KRuns): T and its gradients, zero for samples outside the
// window.  The (win + 1)^2 image and gradient footprint is first staged in
// shared memory (16-byte cp.async chunks of each clamped row when the
// columns lie inside the level -- they may read up to 26 image bytes (window
// 21; at most 30 for any window) and 24 gradient bytes past a row's last
// pixel, inside the pitch, the pyramid allocation's slack, or the 32 bytes a
// caller-owned level 0 keeps readable after its last row -- else one clamped
// column per lane; computed in place for a level without gradient planes).
template <int WIN, int GT>
__device__ __forceinline__ void load_template(const Level &L, float ux, float uy, int lane,
                                              float (&T)[KRuns<WIN>::NS], float (&GX)[KRuns<WIN>::NS],
                                              float (&GY)[KRuns<WIN>::NS], KSmem<WIN> &sm, int &offi, int &offg) {
    constexpr int HW = WIN / 2;
    constexpr int NC = KSmem<WIN>::NC, JS = KSmem<WIN>::JS, NG = KSmem<WIN>::NG, GS = KSmem<WIN>::GS;
    constexpr int RL = KRuns<WIN>::RL, RPL = KRuns<WIN>::RPL;
    // staged gradient words are int16 pairs when computed in place
    constexpr int GTS = GT == VT_GRAD_NONE ? VT_GRAD_S16 : GT;
    const float fx = floorf(ux), fy = floorf(uy);
    const float ax = ux - fx, ay = uy - fy;
    const int x0 = (int)fx - HW, y0 = (int)fy - HW;
    const int hm1 = L.h - 1;
    __syncwarp();
    if constexpr (GT == VT_GRAD_NONE) {
        offi = offg = 0;
        stage_window_otf<WIN>(L, x0, y0, lane, sm);
    } else {
        if (x0 >= 0 && x0 + WIN < L.w) {
            const int wx = x0 & ~15, gw = x0 & ~3;
            offi = x0 - wx;
            offg = x0 - gw;
            const uint32_t sbj = (uint32_t)__cvta_generic_to_shared(sm.j);
            const uint32_t sbg = (uint32_t)__cvta_generic_to_shared(sm.g);
            for (int k = lane; k < (WIN + 1) * NC; k += 32) {
                const int row = k / NC, c = k - row * NC;
                const uint8_t *src = L.img + (size_t)clampi(y0 + row, 0, hm1) * L.pitch + wx + 16 * c;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sbj + row * JS + 16 * c), "l"(src)
                             : "memory");
            }
            for (int k = lane; k < (WIN + 1) * NG; k += 32) {
                const int row = k / NG, c = k - row * NG;
                const uint32_t *src = L.grad + (size_t)clampi(y0 + row, 0, hm1) * L.gpitch + gw + 4 * c;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sbg + 4 * (row * GS + 4 * c)),
                             "l"(src)
                             : "memory");
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
        } else {
            offi = offg = 0;
            if (lane <= WIN) {
                const int c = clampi(x0 + lane, 0, L.w - 1);
#pragma unroll
                for (int r = 0; r <= WIN; ++r) {
                    const int row = clampi(y0 + r, 0, hm1);
                    sm.j[r * JS + lane] = __ldg(L.img + (size_t)row * L.pitch + c);
                    sm.g[r * GS + lane] = __ldg(L.grad + (size_t)row * L.gpitch + c);
                }
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        int c, r0;
        bool valid;
        run_of<WIN>(lane, i, c, r0, valid);
        const uint8_t *jr = valid ? &sm.j[r0 * JS + offi + c] : sm.zj;
        const uint32_t *gr = valid ? &sm.g[r0 * GS + offg + c] : sm.zg;
        float pi = 0.f, pgx = 0.f, pgy = 0.f;
#pragma unroll
        for (int r = 0; r <= RL; ++r) {
            const float mv = u8f(jr[r * JS]), mvr = u8f(jr[r * JS + 1]);
            float gx, gy, gxr, gyr;
            unpack_grad<GTS>(gr[r * GS], gx, gy);
            unpack_grad<GTS>(gr[r * GS + 1], gxr, gyr);
            const float hi = fmaf(ax, mvr - mv, mv);
            const float hgx = fmaf(ax, gxr - gx, gx);
            const float hgy = fmaf(ax, gyr - gy, gy);
            if (r > 0) {
                T[i * RL + r - 1] = fmaf(ay, hi - pi, pi);  // zero for a run outside the window
                GX[i * RL + r - 1] = fmaf(ay, hgx - pgx, pgx);
                GY[i * RL + r - 1] = fmaf(ay, hgy - pgy, pgy);
            }
            pi = hi;
            pgx = hgx;
            pgy = hgy;
        }
    }
}

// Stage the (win + 1) x (win + 1) footprint of J with top-left (x0, y0) in
// shared memory, rows and columns clamped into the image (replicate).  When
// its columns lie inside the image, each (clamped) row is copied in whole
// aligned 16-byte chunks by cp.async (global to shared, no register round
// trip); they may read up to 26 bytes (window 21) past a row's last pixel,
// inside the level's pitch, the pyramid allocation's slack or a caller-owned
// level 0's 32 readable bytes after its last row.  Otherwise lane
// c loads column c (clamped) of every row.  Returns the byte offset of column
// 0 within a staged row.
template <int WIN>
__device__ __forceinline__ int stage_footprint(const Level &L, int x0, int y0, int lane, KSmem<WIN> &sm) {
    constexpr int NC = KSmem<WIN>::NC, JS = KSmem<WIN>::JS;
    int off;
    __syncwarp();  // every lane is done with the previous footprint
    if (x0 >= 0 && x0 + WIN < L.w) {
        const int wx0 = x0 & ~15;
        off = x0 - wx0;
        const uint8_t *base = L.img + wx0;
        const int hm1 = L.h - 1;
        const uint32_t sb = (uint32_t)__cvta_generic_to_shared(sm.j);
        for (int k = lane; k < (WIN + 1) * NC; k += 32) {
            const int row = k / NC, wc = k - row * NC;
            const uint8_t *g = base + (size_t)clampi(y0 + row, 0, hm1) * L.pitch + 16 * wc;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sb + row * JS + 16 * wc), "l"(g) : "memory");
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    } else {
        off = 0;
        if (lane <= WIN) {
            const uint8_t *col = L.img + clampi(x0 + lane, 0, L.w - 1);
            const int hm1 = L.h - 1;
#pragma unroll
            for (int r = 0; r <= WIN; ++r) sm.j[r * JS + lane] = __ldg(col + (size_t)clampi(y0 + r, 0, hm1) * L.pitch);
        }
    }
    __syncwarp();
    return off;
}

// Moments of one integer footprint F (top-left (x0, y0)) against the template.
// With F00 = F(y, x), F01 = F(y, x+1), F10 = F(y+1, x), F11 = F(y+1, x+1) for
// window sample (y, x), the bilinear sample at fractional offset (bx, by) is
//   F00 + bx (F01 - F00) + by (F10 - F00) + bx by (F11 - F10 - F01 + F00),
// so for every q with floor(q) = (x0, y0) + (h, h):
//   sum r grad T = R - bx Sx - by Sy - bx by Sxy,
//   R = sum (T - F00) grad T, Sx = sum (F01 - F00) grad T,
//   Sy = sum (F10 - F00) grad T, Sxy = sum (F11 - F10 - F01 + F00) grad T.
// The footprint differences are exact (integers); m[0..3] are the x parts
// (R, Sx, Sy, Sxy against Tx), m[4..7] the y parts.
template <int WIN>
__device__ __forceinline__ void cell_moments(const Level &L, int x0, int y0, int lane,
                                             const float (&T)[KRuns<WIN>::NS], const float (&GX)[KRuns<WIN>::NS],
                                             const float (&GY)[KRuns<WIN>::NS], KSmem<WIN> &sm, float (&m)[8]) {
    constexpr int JS = KSmem<WIN>::JS, RL = KRuns<WIN>::RL, RPL = KRuns<WIN>::RPL;
    const int off = stage_footprint<WIN>(L, x0, y0, lane, sm);
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.f;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        int c, r0;
        bool valid;
        run_of<WIN>(lane, i, c, r0, valid);  // samples of a run outside the window weigh zero
        const uint8_t *jr = &sm.j[r0 * JS + off + c];
        float pmv = 0.f, pdx = 0.f;
#pragma unroll
        for (int r = 0; r <= RL; ++r) {
            const float mv = u8f(jr[r * JS]);
            const float dx = u8f(jr[r * JS + 1]) - mv;  // F(r, c+1) - F(r, c), exact
            if (r > 0) {
                const int s = i * RL + r - 1;
                const float e0 = T[s] - pmv;
                const float sy = mv - pmv;   // F10 - F00
                const float sxy = dx - pdx;  // F11 - F10 - F01 + F00
                const float gx = GX[s], gy = GY[s];
                a[0] = fmaf(e0, gx, a[0]);
                a[1] = fmaf(pdx, gx, a[1]);
                a[2] = fmaf(sy, gx, a[2]);
                a[3] = fmaf(sxy, gx, a[3]);
                a[4] = fmaf(e0, gy, a[4]);
                a[5] = fmaf(pdx, gy, a[5]);
                a[6] = fmaf(sy, gy, a[6]);
                a[7] = fmaf(sxy, gy, a[7]);
            }
            pmv = mv;
            pdx = dx;
        }
    }
    warp_sum8(a, lane, m);
}

// Error sweep at (qx, qy): sum |T - J_l(q + x)| over the window.
template <int WIN>
__device__ __forceinline__ float abs_residual(const Level &L, float qx, float qy, int lane,
                                              const float (&T)[KRuns<WIN>::NS], KSmem<WIN> &sm) {
    constexpr int HW = WIN / 2, JS = KSmem<WIN>::JS, RL = KRuns<WIN>::RL, RPL = KRuns<WIN>::RPL;
    const float fx = floorf(qx), fy = floorf(qy);
    const float bx = qx - fx, by = qy - fy;
    const int off = stage_footprint<WIN>(L, (int)fx - HW, (int)fy - HW, lane, sm);
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        int c, r0;
        bool valid;
        run_of<WIN>(lane, i, c, r0, valid);
        const uint8_t *jr = valid ? &sm.j[r0 * JS + off + c] : sm.zj;
        float ph = 0.f;
#pragma unroll
        for (int r = 0; r <= RL; ++r) {
            const float mv = u8f(jr[r * JS]);
            const float h = fmaf(bx, u8f(jr[r * JS + 1]) - mv, mv);
            if (r > 0) {
                const float jv = fmaf(by, h - ph, ph);
                const float e = fabsf(T[i * RL + r - 1] - jv);  // 0 - 0 for a run outside the window
                if (r & 1)
                    sa += e;
                else
                    sb += e;
            }
            ph = h;
        }
    }
    return warp_sum(sa + sb);
}

// ---------------------------------------------------------------------------
// FP64 levels.  Where the gradient matrix of a level's template is
// ill-conditioned (lambda_max / lambda_min above kFp64Cond), the FP32 sums of
// G and b lose the weak direction: their rounding, divided by lambda_min,
// moves the Newton steps along it by more than the flow tolerance.  Such a
// level is tracked in FP64: the template and its gradients are sampled in
// FP64 from the staged windows (kept in sm.t / sm.g) at every sweep, G, the
// footprint moments, the 2x2 solve and the position update are FP64.  The
// branch is warp-uniform; with the default eigenvalue threshold (1e-4) an
// accepted template cannot exceed a condition number of 5e3 (fp64_needed),
// so it is taken only when a caller lowers the threshold.

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
    return v;
}

// Keep the template's image window: copy sm.j (as staged by load_template)
// to sm.t before footprints overwrite it.
template <int WIN>
__device__ __forceinline__ void keep_template_window(int lane, KSmem<WIN> &sm) {
    constexpr int NB = (WIN + 1) * KSmem<WIN>::JS / 16;
    __syncwarp();
    const uint4 *src = reinterpret_cast<const uint4 *>(sm.j);
    uint4 *dst = reinterpret_cast<uint4 *>(sm.t);
    for (int k = lane; k < NB; k += 32) dst[k] = src[k];
    __syncwarp();
}

// The lane's samples of one staged template row pair in FP64: horizontal
// lerps of row r of the template image and gradient windows.
template <int WIN, int GT>
__device__ __forceinline__ void tmpl_row64(const uint8_t *tr, const uint32_t *gr, int r, double ax, double unit,
                                           double &hT, double &hGX, double &hGY) {
    constexpr int JS = KSmem<WIN>::JS, GS = KSmem<WIN>::GS;
    constexpr int GTS = GT == VT_GRAD_NONE ? VT_GRAD_S16 : GT;
    const double t0 = (double)tr[r * JS], t1 = (double)tr[r * JS + 1];
    float gx0, gy0, gx1, gy1;
    unpack_grad<GTS>(gr[r * GS], gx0, gy0);
    unpack_grad<GTS>(gr[r * GS + 1], gx1, gy1);
    const double x0 = (double)gx0 * unit, x1 = (double)gx1 * unit, y0 = (double)gy0 * unit, y1 = (double)gy1 * unit;
    hT = fma(ax, t1 - t0, t0);
    hGX = fma(ax, x1 - x0, x0);
    hGY = fma(ax, y1 - y0, y0);
}

// G of the level's template in FP64 (grey levels per pixel), every lane
// holding the totals.
template <int WIN, int GT>
__device__ __forceinline__ void template_G64(double ax, double ay, int offi, int offg, int lane, const KSmem<WIN> &sm,
                                             double &g11, double &g12, double &g22) {
    constexpr int JS = KSmem<WIN>::JS, GS = KSmem<WIN>::GS, RL = KRuns<WIN>::RL, RPL = KRuns<WIN>::RPL;
    constexpr double unit = (double)grad_unit<GT>();
    double a11 = 0.0, a12 = 0.0, a22 = 0.0;
#pragma unroll 1
    for (int i = 0; i < RPL; ++i) {
        int c, r0;
        bool valid;
        run_of<WIN>(lane, i, c, r0, valid);
        if (!valid) continue;
        const uint8_t *tr = &sm.t[r0 * JS + offi + c];
        const uint32_t *gr = &sm.g[r0 * GS + offg + c];
        double pT, pX, pY;
        tmpl_row64<WIN, GT>(tr, gr, 0, ax, unit, pT, pX, pY);
#pragma unroll 1
        for (int r = 1; r <= RL; ++r) {
            double hT, hX, hY;
            tmpl_row64<WIN, GT>(tr, gr, r, ax, unit, hT, hX, hY);
            const double gx = fma(ay, hX - pX, pX), gy = fma(ay, hY - pY, pY);
            a11 = fma(gx, gx, a11);
            a12 = fma(gx, gy, a12);
            a22 = fma(gy, gy, a22);
            pT = hT;
            pX = hX;
            pY = hY;
        }
    }
    g11 = warp_sum_d(a11);
    g12 = warp_sum_d(a12);
    g22 = warp_sum_d(a22);
}

// The eight footprint moments of cell_moments in FP64, the template sampled
// in FP64 from the kept windows (grey levels per pixel).
template <int WIN, int GT>
__device__ __forceinline__ void cell_moments64(const Level &L, int x0, int y0, double ax, double ay, int offi,
                                               int offg, int lane, KSmem<WIN> &sm, double (&m)[8]) {
    constexpr int JS = KSmem<WIN>::JS, GS = KSmem<WIN>::GS, RL = KRuns<WIN>::RL, RPL = KRuns<WIN>::RPL;
    constexpr double unit = (double)grad_unit<GT>();
    const int off = stage_footprint<WIN>(L, x0, y0, lane, sm);
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.0;
#pragma unroll 1
    for (int i = 0; i < RPL; ++i) {
        int c, r0;
        bool valid;
        run_of<WIN>(lane, i, c, r0, valid);
        if (!valid) continue;
        const uint8_t *tr = &sm.t[r0 * JS + offi + c];
        const uint32_t *gr = &sm.g[r0 * GS + offg + c];
        const uint8_t *jr = &sm.j[r0 * JS + off + c];
        double pT, pX, pY;
        tmpl_row64<WIN, GT>(tr, gr, 0, ax, unit, pT, pX, pY);
        double pmv = (double)jr[0];
        double pdx = (double)jr[1] - pmv;
#pragma unroll 1
        for (int r = 1; r <= RL; ++r) {
            double hT, hX, hY;
            tmpl_row64<WIN, GT>(tr, gr, r, ax, unit, hT, hX, hY);
            const double T = fma(ay, hT - pT, pT), gx = fma(ay, hX - pX, pX), gy = fma(ay, hY - pY, pY);
            const double mv = (double)jr[r * JS];
            const double dx = (double)jr[r * JS + 1] - mv;
            const double e0 = T - pmv, sy = mv - pmv, sxy = dx - pdx;
            a[0] = fma(e0, gx, a[0]);
            a[1] = fma(pdx, gx, a[1]);
            a[2] = fma(sy, gx, a[2]);
            a[3] = fma(sxy, gx, a[3]);
            a[4] = fma(e0, gy, a[4]);
            a[5] = fma(pdx, gy, a[5]);
            a[6] = fma(sy, gy, a[6]);
            a[7] = fma(sxy, gy, a[7]);
            pT = hT;
            pX = hX;
            pY = hY;
            pmv = mv;
            pdx = dx;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k] = warp_sum_d(a[k]);
}

// Result of one FP64 level.
struct Level64 {
    double nx, ny;  // step sum from the level's guess
    float lmin;     // normalised lambda_min (FP64, rounded)
    int reason;     // VT_TRACKED, VT_LOST_EIG or VT_LOST_OOB
    int iters, sweeps;
};

// One level in FP64 (see kFp64Cond): the eigenvalue test and the Newton
// iterations from the level's guess (gx, gy).
template <int WIN, int GT>
__device__ __forceinline__ Level64 track_level64(const Level Jl, const int max_iters, const float eps2,
                                              const float min_eig, float ux, float uy, float gx, float gy, int offi,
                                              int offg, int lane, KSmem<WIN> *smp) {
    constexpr int HW = WIN / 2;
    constexpr double N = (double)(WIN * WIN);
    KSmem<WIN> &sm = *smp;
    Level64 o;
    o.reason = VT_TRACKED;
    o.iters = 0;
    o.sweeps = 0;
    o.nx = o.ny = 0.0;
    keep_template_window<WIN>(lane, sm);
    const double ax = (double)(ux - floorf(ux)), ay = (double)(uy - floorf(uy));
    double G11, G12, G22;
    template_G64<WIN, GT>(ax, ay, offi, offg, lane, sm, G11, G12, G22);
    const double det64 = G11 * G22 - G12 * G12;
    const double lmax64 = 0.5 * (G11 + G22 + sqrt((G11 - G22) * (G11 - G22) + 4.0 * G12 * G12));
    const double lmin64 = det64 / lmax64 / (N * 65025.0);
    o.lmin = (float)lmin64;
    if (!(lmin64 >= (double)min_eig) || !(det64 > 0.0)) {
        o.reason = VT_LOST_EIG;
        return o;
    }
    int cx = INT_MIN, cy = INT_MIN;
    double m[8];
    const double uxd = (double)ux + (double)gx, uyd = (double)uy + (double)gy;
    for (int k = 0; k < max_iters; ++k) {
        const double qx = uxd + o.nx, qy = uyd + o.ny;
        const double dist = fmin(fmin(qx + (double)HW, (double)(Jl.w - 1 + HW) - qx),
                                 fmin(qy + (double)HW, (double)(Jl.h - 1 + HW) - qy));
        if (!(dist >= 0.0)) {
            o.reason = VT_LOST_OOB;
            return o;
        }
        const double fx = floor(qx), fy = floor(qy);
        const int ix = (int)fx - HW, iy = (int)fy - HW;
        if (ix != cx || iy != cy) {
            cell_moments64<WIN, GT>(Jl, ix, iy, ax, ay, offi, offg, lane, sm, m);
            cx = ix;
            cy = iy;
            ++o.sweeps;
        }
        const double bx = qx - fx, by = qy - fy, bxy = bx * by;
        const double b1 = m[0] - bx * m[1] - by * m[2] - bxy * m[3];
        const double b2 = m[4] - bx * m[5] - by * m[6] - bxy * m[7];
        const double ex = (G22 * b1 - G12 * b2) / det64;
        const double ey = (G11 * b2 - G12 * b1) / det64;
        o.nx += ex;
        o.ny += ey;
        ++o.iters;
        if (ex * ex + ey * ey < (double)eps2) break;
    }
    return o;
}

// Internal reason of a point the FP32 tracker leaves to the FP64-capable one
// (its status is written as kStatusPending until that second launch).
constexpr int kReasonPending = 255;
constexpr uint8_t kStatusPending = 2;

// Track one point u = (ux0, uy0) from pyramid I to pyramid J.  The FP32
// tracker (F64 = false) stops at a level whose template is ill-conditioned
// (kFp64Cond) and marks the point pending (kReasonPending); the kernels then
// leave it to a second, FP64-capable launch (F64 = true) that tracks it again
// from the start with such levels in FP64.  Levels are deterministic, so its
// coarser levels give the same results the second time.  Keeping the FP64
// code out of the FP32 kernels keeps their registers free of it.
template <int WIN, int GT, bool F64>
__device__ __forceinline__ void track_point(const Level *I, const Level *J, const KParams &P, float ux0, float uy0,
                                            bool has_guess, float gux, float guy, int lane, KSmem<WIN> &sm, KOut &o,
                                            bool want_err) {
    constexpr int HW = WIN / 2;
    constexpr float N = (float)(WIN * WIN);
    constexpr float unit = grad_unit<GT>();
    // lambda_min normalisation: stored units^2 -> (grey/px)^2, / (N 255^2)
    const float inv_norm = unit * unit / (N * 65025.0f);
    constexpr int NS = KRuns<WIN>::NS;
    float T[NS], GX[NS], GY[NS];
    const int L = P.levels;
    float gx = 0.f, gy = 0.f, nux = 0.f, nuy = 0.f;
    double nx64 = 0.0, ny64 = 0.0;  // the step sum of an FP64 level
    bool level64 = false;           // the last level examined ran in FP64
    int lost_level = 0;
    o.status = 1;
    o.reason = VT_TRACKED;
    o.iters = 0;
    o.tmpl = 0;
    o.errp = 0;
    o.sweeps = 0;
    o.err = 0.f;
    o.lmin = __int_as_float(0x7fc00000);
    if (!(ux0 >= 0.f && ux0 <= (float)(I[0].w - 1) && uy0 >= 0.f && uy0 <= (float)(I[0].h - 1))) {
        o.status = 0;
        o.reason = VT_LOST_INPUT;
        o.x = ux0;
        o.y = uy0;
        return;
    }
    if (has_guess) {
        const float s = pow2neg(L - 1);
        gx = (gux - ux0) * s;
        gy = (guy - uy0) * s;
    }
    for (int l = L - 1; l >= 0; --l) {
        // by value: the fields stay in registers across the staging copies
        const Level Il = I[l];
        const Level Jl = J[l];
        const float s = pow2neg(l);
        const float ux = ux0 * s, uy = uy0 * s;
        int offi, offg;
        load_template<WIN, GT>(Il, ux, uy, lane, T, GX, GY, sm, offi, offg);
        ++o.tmpl;
        float a11 = 0.f, a12 = 0.f, a22 = 0.f;
#pragma unroll
        for (int r = 0; r < NS; ++r) {
            a11 = fmaf(GX[r], GX[r], a11);
            a12 = fmaf(GX[r], GY[r], a12);
            a22 = fmaf(GY[r], GY[r], a22);
        }
        float g11, g12, g22;
        warp_sum3(a11, a12, a22, lane, g11, g12, g22);
        // lambda_min = det / lambda_max avoids the cancellation of (tr - disc) / 2
        const float tr = g11 + g22, df = g11 - g22;
        const float lmax = 0.5f * (tr + sqrtf(fmaf(df, df, 4.f * g12 * g12)));
        const float det = kdiff(g11, g22, g12, g12);  // sign exact, 2 ulp
        const float lmin = det / lmax;
        o.lmin = lmin * inv_norm;
        nux = nuy = 0.f;
        // ill-conditioned (or det <= 0): decided and tracked in FP64
        level64 = P.fp64 && !(lmin * kFp64Cond >= lmax);
        if (level64) {
            if constexpr (!F64) {
                o.status = 0;
                o.reason = kReasonPending;
                return;
            } else {
                const Level64 r = track_level64<WIN, GT>(Jl, P.max_iters, P.eps2, P.min_eig, ux, uy, gx, gy, offi,
                                                         offg, lane, &sm);
                o.lmin = r.lmin;
                o.iters += r.iters;
                o.sweeps += r.sweeps;
                nx64 = r.nx;
                ny64 = r.ny;
                if (r.reason != VT_TRACKED) {
                    o.status = 0;
                    o.reason = r.reason;
                    lost_level = l;
                    break;
                }
                if (l > 0) {
                    gx = (float)(2.0 * ((double)gx + nx64));
                    gy = (float)(2.0 * ((double)gy + ny64));
                    level64 = false;
                }
                continue;
            }
        }
        if (!(o.lmin >= P.min_eig) || !(det > 0.f)) {
            o.status = 0;
            o.reason = VT_LOST_EIG;
            lost_level = l;
            break;
        }
        // eta = G^-1 b in grey/px units: G = unit^2 G_s, b = unit b_s => eta = adj(G_s) b_s / (unit det_s)
        // (unit is a power of two, so det * unit is exact; the adjugate
        // products cancel for ill-conditioned G, hence kdiff)
        const float inv_det = 1.0f / (det * unit);
        // moments of the footprint cell last swept (valid while the integer
        // part of q does not change)
        int cx = INT_MIN, cy = INT_MIN;
        float m[8];
        for (int k = 0; k < P.max_iters; ++k) {
            const float qx = ux + gx + nux, qy = uy + gy + nuy;
            const float dist = fminf(fminf(qx + (float)HW, (float)(Jl.w - 1 + HW) - qx),
                                     fminf(qy + (float)HW, (float)(Jl.h - 1 + HW) - qy));
            if (!(dist >= 0.f)) {
                o.status = 0;
                o.reason = VT_LOST_OOB;
                break;
            }
            const float fx = floorf(qx), fy = floorf(qy);
            const int ix = (int)fx - HW, iy = (int)fy - HW;
            if (ix != cx || iy != cy) {
                cell_moments<WIN>(Jl, ix, iy, lane, T, GX, GY, sm, m);
                cx = ix;
                cy = iy;
                ++o.sweeps;
            }
            const float bx = qx - fx, by = qy - fy, bxy = bx * by;
            const float b1 = m[0] - bx * m[1] - by * m[2] - bxy * m[3];
            const float b2 = m[4] - bx * m[5] - by * m[6] - bxy * m[7];
            const float ex = kdiff(g22, b1, g12, b2) * inv_det;
            const float ey = kdiff(g11, b2, g12, b1) * inv_det;
            nux += ex;
            nuy += ey;
            ++o.iters;
            if (ex * ex + ey * ey < P.eps2) break;
        }
        if (!o.status) {
            lost_level = l;
            break;
        }
        if (l > 0) {
            gx = 2.f * (gx + nux);
            gy = 2.f * (gy + nuy);
        }
    }
    {
        const float sc = (float)(1 << lost_level);
        const float si = pow2neg(lost_level);
        if (F64 && level64) {
            o.x = (float)(((double)(ux0 * si) + (double)gx + nx64) * (double)sc);
            o.y = (float)(((double)(uy0 * si) + (double)gy + ny64) * (double)sc);
        } else {
            o.x = (ux0 * si + gx + nux) * sc;
            o.y = (uy0 * si + gy + nuy) * sc;
        }
    }
    if (o.status) {
        const float dist = fminf(fminf(o.x, (float)(I[0].w - 1) - o.x), fminf(o.y, (float)(I[0].h - 1) - o.y));
        if (!(dist >= 0.f)) {
            o.status = 0;
            o.reason = VT_LOST_OOB;
        } else {
            // T still holds level 0's template
            if (want_err) {
                o.err = abs_residual<WIN>(J[0], o.x, o.y, lane, T, sm) / N;
                ++o.errp;
            }
        }
    }
}

// Forward I->J (pass 0) and, with fb, backward J->I from the forward result
// (pass 1) followed by the FB test.  One inlined copy of track_point serves
// both passes, and every kernel (single-pair or batched) calls this function,
// so a point's result does not depend on which kernel tracked it.
template <int WIN, int GT, bool F64>
__device__ __forceinline__ void track_point_dir(const Level *I, const Level *J, const KParams &P, float ux0,
                                                float uy0, bool fb, bool has_guess, float gux, float guy, int lane,
                                                KSmem<WIN> &sm, KOut &o) {
    const Level *A = I, *B = J;
    float x = ux0, y = uy0;
    const int npass = fb ? 2 : 1;
#pragma unroll 1
    for (int pass = 0; pass < npass; ++pass) {
        KOut r;
        // the backward pass only decides the status: its error is not an output
        track_point<WIN, GT, F64>(A, B, P, x, y, pass == 0 && has_guess, gux, guy, lane, sm, r, pass == 0);
        if (pass == 0) {
            o = r;
            if (!r.status) return;
            x = r.x;
            y = r.y;
            A = J;
            B = I;
        } else {
            o.iters += r.iters;
            o.tmpl += r.tmpl;
            o.errp += r.errp;
            o.sweeps += r.sweeps;
            if (!r.status) {
                o.status = 0;
                o.reason = r.reason;
                return;
            }
            const float dx = ux0 - r.x, dy = uy0 - r.y;
            if (!(dx * dx + dy * dy <= P.fb_thr2)) {
                o.status = 0;
                o.reason = VT_LOST_FB;
            }
        }
    }
}

}  // namespace vt
