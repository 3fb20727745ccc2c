// Shi-Tomasi (GFTT) corner detection (K6) on pyramid levels of one or many
// frames at once (the classical detector the paper pairs with LK tracking,
// Sec. IV; run on the CPU in the paper, Sec. V-F).  It reuses the levels'
// stored int16 Scharr gradients.  Every launch covers every frame ("job") of
// the call:
//
//   K6a k_gftt_local   per tile: the gradient words (reflect-101 borders) in
//                      shared memory; a, b, c = (2br+1)^2 box sums of gx^2,
//                      gx gy, gy^2 (exact integers) and lambda_min in FP32 with
//                      explicit round-to-nearest operations, clamped at 0, for
//                      the tile and an nms halo; the frame maximum (one atomic
//                      per tile); every pixel outside the border that is the
//                      maximum of its (2nms+1)^2 window (separable maximum;
//                      ties to the smaller index) and not within min_dist of a
//                      mask point (a byte map the mask kernel rasterises with
//                      the same FP32 test) is a local maximum: a 64-bit key
//                      (score bits, ~pixel).
//   K6b k_gftt_filter  local maxima with lambda >= quality * max: the frame's
//                      candidates.
//   K6c first pass     per frame (one CTA, k_gftt_greedy_top): the candidates
//                      of the smallest set of top score-histogram bins holding
//                      a few times max_corners of them, sorted in shared
//                      memory, then a warp's greedy min-distance pass in
//                      priority order -- the greedy's decisions depend only on
//                      higher-priority candidates, so its first max_corners
//                      kept are the full greedy's.
//   K6d second pass    frames the first pass could not settle (fewer kept than
//                      max_corners while more candidates exist, or too many
//                      participants): a counting sort of all candidates into
//                      cells at least min_dist wide, the greedy resolved in
//                      parallel rounds over the cells (k_gftt_select:
//                      cooperative launch, a grid-wide barrier per round), and
//                      k_gftt_output ordering the kept (a score-histogram top
//                      set sorted in shared memory, or a bitonic sort of all
//                      kept in global memory).
// Every decision is taken on the same FP32 values the oracle computes, so the
// corner lists are exact.
#include <cooperative_groups.h>

#include <cstdint>
#include <cstdlib>

#include "vt_internal.cuh"

namespace cg = cooperative_groups;

namespace vt {

constexpr int GF_TX = 64, GF_TY = 16;  // score / local-maximum tiles
constexpr int GF_MAX_BR = 3, GF_MAX_NMS = 8;
constexpr int GF_OUT_THREADS = 1024;
constexpr int GF_SCAN_THREADS = 1024;
constexpr int GF_MIS_THREADS = 256;
constexpr int GF_SMEM_SORT = 16384;  // keys sorted in shared memory (128 KB)
constexpr int GF_HIST = 4096;        // score-bit histogram bins of the output kernel
constexpr int GF_MAX_CORNERS = 8192;
constexpr int GF_GRID_THREADS = 256;
constexpr int kMaxGfttJobs = 64;
// The selection first runs over the candidates of the smallest set of top
// score-histogram bins holding at least GF_TOP_FACTOR * max_corners (and at
// least GF_TOP_MIN) of them; only if that leaves fewer than max_corners kept
// does it run again over every candidate.
constexpr int GF_TOP_FACTOR = 4, GF_TOP_MIN = 512;
constexpr int GF_TOP_MAX = 2048;    // first-pass participants (a warp's greedy); more go to the second pass
constexpr int GF_GR_CELLS = 16384;  // first-pass cell grid
constexpr int GF_GR_THREADS = 1024;
struct GreedySmem {
    unsigned long long key[GF_TOP_MAX];
    uint32_t pxy[GF_TOP_MAX];  // (x, y) of the sorted participants
    int head[GF_GR_CELLS];
    int16_t next[GF_MAX_CORNERS];
    uint32_t kxy[GF_MAX_CORNERS];
    int n;
};
enum : uint8_t { GF_UNDECIDED = 0, GF_KEPT = 1, GF_REJECTED = 2 };

struct GJob {
    const uint32_t *grad;
    int gpitch, w, h;
    int tiles_x, tile0;  // score / candidate tiles of this frame, first tile
    int px0;             // first pixel of this frame in the concatenated buffers
    int cell0, cells_x, cells_y;  // cell grid (cell0: first of cells_x * cells_y + 1 entries)
    long long kept0;              // kept segment (a power of two >= w h entries)
    int kept_cap;
    const float2 *mask;
    int n_mask;
    float2 *out;
    float *out_score;
    int *out_count;
    int max_corners;
    int gr_cell, gr_cx, gr_cy;  // cell grid of the first-pass greedy (cells >= min_dist, <= GF_GR_CELLS)
};

struct GJobs {
    int n, tiles, br, nms, border, min_dist;
    float quality;
    GJob j[kMaxGfttJobs];
};

// Per-frame counters in the workspace.
struct GCount {
    unsigned maxbits;  // maximum score bits
    int lmax;          // local maxima (before the quality threshold)
    int cand;          // candidates
    int part;          // candidates taking part in the selection (keys >= lo)
    int kept;          // kept by the selection
    int retry;         // the top set was too small: select again over every candidate
    unsigned long long lo;
};

// a, b, c fit in 32 bits (at most 49 * 4080^2), so their conversions to float
// round exactly like the oracle's 64-bit ones.
__device__ __forceinline__ float gftt_score(int a, int b, int c) {
    const float fa = (float)a, fb = (float)b, fc = (float)c;
    const float d = __fsub_rn(fa, fc);
    const float q = __fadd_rn(__fmul_rn(d, d), __fmul_rn(4.0f, __fmul_rn(fb, fb)));
    const float t = __fsub_rn(__fadd_rn(fa, fc), __fsqrt_rn(q));
    const float l = __fmul_rn(0.5f, t);
    return l > 0.0f ? l : 0.0f;
}

__device__ __forceinline__ int tile_job(const GJobs &J, int t) {
    int lo = 0, hi = J.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (J.j[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ unsigned key_pixel(unsigned long long k) { return 0xffffffffu - (unsigned)(k & 0xffffffffu); }

// Pixels within min_dist of a mask point, marked in a byte map (one warp per
// mask point, blockIdx.y: frame).  The test is the candidate test itself,
// (x - px)^2 + (y - py)^2 < min_dist^2 in single precision, evaluated over a
// box one pixel wider than the disc, so the map is exact.
__global__ void k_gftt_mask(const __grid_constant__ GJobs J, uint8_t *masked) {
    const GJob &G = J.j[blockIdx.y];
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int md = J.min_dist;
    const float md2 = (float)(md * md);
    uint8_t *mp = masked + G.px0;
    for (int m = blockIdx.x * wpb + (threadIdx.x >> 5); m < G.n_mask; m += gridDim.x * wpb) {
        const float2 p = G.mask[m];
        if (!(p.x > -(float)(md + 2) && p.x < (float)(G.w + md + 2) && p.y > -(float)(md + 2) &&
              p.y < (float)(G.h + md + 2)))
            continue;  // non-finite or too far away to mask a pixel
        const int x0 = max(0, (int)floorf(p.x) - md - 1), x1 = min(G.w - 1, (int)ceilf(p.x) + md + 1);
        const int y0 = max(0, (int)floorf(p.y) - md - 1), y1 = min(G.h - 1, (int)ceilf(p.y) + md + 1);
        const int bw = x1 - x0 + 1;
        for (int k = lane; k < bw * (y1 - y0 + 1); k += 32) {
            const int y = y0 + k / bw, x = x0 + k % bw;
            const float dx = __fsub_rn((float)x, p.x), dy = __fsub_rn((float)y, p.y);
            if (__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) < md2) mp[(size_t)y * G.w + x] = 1;
        }
    }
}

// Scores, frame maximum and local maxima in one pass over the gradients
// (one CTA per GF_TX x GF_TY tile of one frame): the gradient words of the
// tile plus an (nms + br) halo (reflect-101) are staged in shared memory, the
// scores of the tile plus an nms halo computed from them (outside the image:
// -1, which never competes), and each output pixel outside the border that
// is the maximum of its window (separable maximum; an equal score at a
// smaller index wins the tie) and not masked goes to the frame's list of
// local maxima.  The quality threshold, which needs the frame maximum, is
// applied afterwards (k_gftt_filter).
template <int BR>  // block radius: the box-sum taps unroll with constant offsets
__global__ void __launch_bounds__(GF_TX *GF_TY) k_gftt_local(const __grid_constant__ GJobs J, GCount *cnt,
                                                             const uint8_t *masked, unsigned long long *lmax) {
    constexpr int HG = GF_MAX_NMS + GF_MAX_BR;
    __shared__ uint32_t sg[GF_TY + 2 * HG][GF_TX + 2 * HG];
    __shared__ float sc[GF_TY + 2 * GF_MAX_NMS][GF_TX + 2 * GF_MAX_NMS];
    __shared__ float rmax[GF_TY + 2 * GF_MAX_NMS][GF_TX];
    __shared__ unsigned wm[GF_TX * GF_TY / 32];
    const int jb = tile_job(J, blockIdx.x);
    const GJob &G = J.j[jb];
    const int t = blockIdx.x - G.tile0, ty = t / G.tiles_x, tx = t - ty * G.tiles_x;
    constexpr int br = BR;
    const int x0 = tx * GF_TX, y0 = ty * GF_TY, nms = J.nms, hg = nms + br;
    const int tid = threadIdx.y * GF_TX + threadIdx.x;
    const int gw = GF_TX + 2 * hg, gh = GF_TY + 2 * hg;
    const bool interior = x0 - hg >= 0 && y0 - hg >= 0 && x0 + GF_TX + hg <= G.w && y0 + GF_TY + hg <= G.h;
    for (int r = threadIdx.y; r < gh; r += GF_TY) {
        const int yy = interior ? y0 + r - hg : refl101(y0 + r - hg, G.h);
        const uint32_t *row = G.grad + (size_t)yy * G.gpitch;
        for (int c = threadIdx.x; c < gw; c += GF_TX)
            sg[r][c] = __ldg(row + (interior ? x0 + c - hg : refl101(x0 + c - hg, G.w)));
    }
    __syncthreads();
    const int sw = GF_TX + 2 * nms, sh = GF_TY + 2 * nms;
    for (int r = threadIdx.y; r < sh; r += GF_TY)
        for (int c = threadIdx.x; c < sw; c += GF_TX) {
        const int yy = y0 + r - nms, xx = x0 + c - nms;
        float v = -1.0f;
        if (yy >= 0 && yy < G.h && xx >= 0 && xx < G.w) {
            int a = 0, b = 0, cc = 0;  // at most 49 * 4080^2 < 2^31
#pragma unroll
            for (int j = 0; j <= 2 * br; ++j)
#pragma unroll
                for (int k = 0; k <= 2 * br; ++k) {
                    const uint32_t g = sg[r + j][c + k];
                    const int u = (int16_t)(g & 0xffffu), w = (int16_t)(g >> 16);
                    a += u * u;
                    b += u * w;
                    cc += w * w;
                }
            v = gftt_score(a, b, cc);
        }
        sc[r][c] = v;
        }
    __syncthreads();
    for (int r = threadIdx.y; r < sh; r += GF_TY) {  // row maxima over each output column's window
        const int c = threadIdx.x;
        float m = sc[r][c];
        for (int k = 1; k <= 2 * nms; ++k) m = fmaxf(m, sc[r][c + k]);
        rmax[r][c] = m;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool inside = x < G.w && y < G.h;
    const float v = inside ? sc[threadIdx.y + nms][threadIdx.x + nms] : 0.0f;
    // frame maximum (scores are >= 0, so their bit patterns order like the values)
    unsigned m = __float_as_uint(v);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) wm[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        unsigned mm = 0;
        for (int k = 0; k < GF_TX * GF_TY / 32; ++k) mm = max(mm, wm[k]);
        atomicMax(&cnt[jb].maxbits, mm);
    }
    const int border = J.border;
    if (!inside || !(v > 0.0f) || x < border || y < border || x >= G.w - border || y >= G.h - border) return;
    float wmax = rmax[threadIdx.y][threadIdx.x];
    for (int k = 1; k <= 2 * nms; ++k) wmax = fmaxf(wmax, rmax[threadIdx.y + k][threadIdx.x]);
    if (wmax > v) return;  // a strictly larger score in the window
    // v is the window maximum: only an equal score at a smaller index can beat it
    for (int j = -nms; j <= 0; ++j)
        for (int i = -nms; i <= nms; ++i) {
            if (j == 0 && i >= 0) break;
            if (sc[threadIdx.y + nms + j][threadIdx.x + nms + i] == v) return;  // (j, i) comes first
        }
    if (G.n_mask > 0 && masked[(size_t)G.px0 + (size_t)y * G.w + x]) return;
    const unsigned gpx = (unsigned)G.px0 + (unsigned)(y * G.w + x);
    const int slot = atomicAdd(&cnt[jb].lmax, 1);
    lmax[(size_t)G.px0 + slot] = ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xffffffffu - gpx);
}

// Local maxima at or above quality * (frame maximum) become the frame's
// candidates (blockIdx.y: frame).
__global__ void k_gftt_filter(const __grid_constant__ GJobs J, GCount *cnt, const unsigned long long *lmax,
                              unsigned long long *keys) {
    const GJob &G = J.j[blockIdx.y];
    GCount &C = cnt[blockIdx.y];
    const int n = C.lmax;
    const float thr = __fmul_rn(J.quality, __uint_as_float(C.maxbits));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long k = lmax[(size_t)G.px0 + i];
        if (__uint_as_float((unsigned)(k >> 32)) >= thr) keys[(size_t)G.px0 + atomicAdd(&C.cand, 1)] = k;
    }
}

// Candidates into cells at least min_dist wide, so every pair closer than
// min_dist lies in neighbouring cells (blockIdx.y: frame).
__global__ void k_gftt_cell_count(const __grid_constant__ GJobs J, const GCount *cnt,
                                  const unsigned long long *keys, int *cell_count, int *rank, int pass) {
    const GJob &G = J.j[blockIdx.y];
    const GCount &C = cnt[blockIdx.y];
    if (pass == 2 && !C.retry) return;
    const int n = C.cand, cs = J.min_dist;
    const unsigned long long lo = C.lo;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[(size_t)G.px0 + i];
        if (k < lo) continue;
        const unsigned p = key_pixel(k) - (unsigned)G.px0;
        const int x = (int)(p % (unsigned)G.w), y = (int)(p / (unsigned)G.w);
        rank[(size_t)G.px0 + i] = atomicAdd(&cell_count[G.cell0 + (y / cs) * G.cells_x + x / cs], 1);
    }
}

// Exclusive scan of each frame's cell counts (one CTA per frame); starts are
// positions in the frame's candidate segment.
__global__ void __launch_bounds__(GF_SCAN_THREADS) k_gftt_cell_scan(const __grid_constant__ GJobs J,
                                                                      const GCount *cnt, int *cell_count,
                                                                      int *cell_start, int pass) {
    __shared__ int part[GF_SCAN_THREADS];
    const GJob &G = J.j[blockIdx.x];
    if (pass == 2 && !cnt[blockIdx.x].retry) return;
    const int ncell = G.cells_x * G.cells_y;
    int *cc = cell_count + G.cell0;
    int *cs = cell_start + G.cell0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int base = G.px0;
    // chunks of 4 consecutive cells per thread (coalesced), scanned with warp shuffles
    for (int c0 = 0; c0 < ncell; c0 += 4 * GF_SCAN_THREADS) {
        const int b = c0 + 4 * threadIdx.x;
        int v[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = b + k < ncell ? cc[b + k] : 0;
            if (b + k < ncell) cc[b + k] = 0;  // clean for the next pass / call
            sum += v[k];
        }
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) part[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = part[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            part[lane] = w;
        }
        __syncthreads();
        int run = base + x - sum + (wid > 0 ? part[wid - 1] : 0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (b + k < ncell) cs[b + k] = run;
            run += v[k];
        }
        base += part[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) cs[ncell] = base;
}

__global__ void k_gftt_cell_scatter(const __grid_constant__ GJobs J, const GCount *cnt,
                                    const unsigned long long *keys, const int *cell_start, const int *rank,
                                    unsigned long long *skeys, uint8_t *state, int pass) {
    const GJob &G = J.j[blockIdx.y];
    const GCount &C = cnt[blockIdx.y];
    if (pass == 2 && !C.retry) return;
    const int n = C.cand, cs = J.min_dist;
    const unsigned long long lo = C.lo;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[(size_t)G.px0 + i];
        if (k < lo) continue;
        const unsigned p = key_pixel(k) - (unsigned)G.px0;
        const int x = (int)(p % (unsigned)G.w), y = (int)(p / (unsigned)G.w);
        const int pos = cell_start[G.cell0 + (y / cs) * G.cells_x + x / cs] + rank[(size_t)G.px0 + i];
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
// (cooperative launch); the kept candidates then go to their frame's kept
// segment.
__global__ void __launch_bounds__(GF_MIS_THREADS) k_gftt_select(const __grid_constant__ GJobs J, GCount *cnt,
                                                                 const unsigned long long *skeys,
                                                                 const int *cell_start, uint8_t *state, int *und,
                                                                 unsigned long long *kept, int pass) {
    cg::grid_group grid = cg::this_grid();
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const long long d2 = (long long)J.min_dist * J.min_dist;
    const int cs = J.min_dist;
    volatile uint8_t *vs = state;
    for (int r = 0;; ++r) {
        if (tid == 0) und[(r + 1) % 3] = 0;  // the slot round r+1 counts into (last read before round r)
        int mine = 0;
        for (int jb = 0; jb < J.n; ++jb) {
            const GJob &G = J.j[jb];
            if (pass == 2 && !cnt[jb].retry) continue;
            const int n = cnt[jb].part;
            for (int q = tid; q < n; q += nth) {
                const int i = G.px0 + q;
                if (vs[i] != GF_UNDECIDED) continue;
                const unsigned long long k = skeys[i];
                const unsigned p = key_pixel(k) - (unsigned)G.px0;
                const int x = (int)(p % (unsigned)G.w), y = (int)(p / (unsigned)G.w);
                const int cx = x / cs, cy = y / cs;
                bool blocked = false, rejected = false;
                for (int dy = -1; dy <= 1 && !rejected; ++dy) {
                    const int yy = cy + dy;
                    if (yy < 0 || yy >= G.cells_y) continue;
                    for (int dx = -1; dx <= 1 && !rejected; ++dx) {
                        const int xx = cx + dx;
                        if (xx < 0 || xx >= G.cells_x) continue;
                        const int c = G.cell0 + yy * G.cells_x + xx;
                        for (int j = cell_start[c], je = cell_start[c + 1]; j < je; ++j) {
                            const unsigned long long kj = skeys[j];
                            if (kj <= k) continue;  // lower priority (or itself)
                            const unsigned pj = key_pixel(kj) - (unsigned)G.px0;
                            const long long ex = (long long)(int)(pj % (unsigned)G.w) - x;
                            const long long ey = (long long)(int)(pj / (unsigned)G.w) - y;
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
        }
        if (mine) atomicAdd(&und[r % 3], mine);
        grid.sync();
        if (*reinterpret_cast<volatile int *>(&und[r % 3]) == 0) break;
    }
    for (int jb = 0; jb < J.n; ++jb) {
        const GJob &G = J.j[jb];
        if (pass == 2 && !cnt[jb].retry) continue;
        const int n = cnt[jb].part;
        for (int q = tid; q < n; q += nth) {
            const int i = G.px0 + q;
            if (vs[i] == GF_KEPT) kept[G.kept0 + atomicAdd(&cnt[jb].kept, 1)] = skeys[i];
        }
    }
}

// Histogram of each frame's candidate keys by their top 12 bits (score
// exponent and three mantissa bits; blockIdx.y: frame).
__global__ void k_gftt_hist(const __grid_constant__ GJobs J, const GCount *cnt, const unsigned long long *keys,
                            int *hist) {
    const GJob &G = J.j[blockIdx.y];
    const int n = cnt[blockIdx.y].cand;
    int *h = hist + (size_t)blockIdx.y * GF_HIST;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&h[(int)(keys[(size_t)G.px0 + i] >> 52)], 1);
}

// The selection's first set per frame: keys >= lo, the smallest set of top
// bins holding the target count (one CTA per frame; thread t holds the four
// bins 4095 - 4t .. 4092 - 4t, a block scan gives the count above them).
__global__ void __launch_bounds__(GF_HIST / 4) k_gftt_top(const __grid_constant__ GJobs J, GCount *cnt,
                                                        const int *hist) {
    __shared__ int wsum[GF_HIST / 4 / 32];
    const GJob &G = J.j[blockIdx.x];
    GCount &C = cnt[blockIdx.x];
    const int target = G.max_corners == 0 ? 0 : max(GF_TOP_FACTOR * G.max_corners, GF_TOP_MIN);
    if (target == 0 || C.cand <= target) {  // nothing to select, or every candidate takes part
        if (threadIdx.x == 0) {
            C.lo = target == 0 ? ~0ull : 0ull;
            C.part = target == 0 ? 0 : C.cand;
        }
        return;
    }
    const int *h = hist + (size_t)blockIdx.x * GF_HIST;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int v[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = h[GF_HIST - 1 - 4 * t - k];
        sum += v[k];
    }
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    int above = x - sum;
    for (int w = 0; w < wid; ++w) above += wsum[w];
    // the bin where the running count (from the top) first reaches the target
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int before = above;
        above += v[k];
        if (before < target && above >= target) {
            C.lo = (unsigned long long)(GF_HIST - 1 - 4 * t - k) << 52;
            C.part = above;
        }
    }
}

// First pass per frame (one CTA): the participants (keys >= lo) sorted in
// shared memory, then one warp runs the greedy in priority order, 32
// candidates at a time: each lane tests its candidate against the kept
// corners through a cell grid in shared memory and forms the mask of the
// earlier lanes of the chunk closer than min_dist; every lane then resolves
// the chunk in order from those masks (kept if no earlier kept lane of the
// chunk conflicts).  The first max_corners kept go straight to the output.
// A frame whose participants keep fewer than max_corners while more
// candidates exist (or whose participants do not fit) is flagged for the
// selection over every candidate (the second pass).
__global__ void __launch_bounds__(GF_GR_THREADS) k_gftt_greedy_top(const __grid_constant__ GJobs J, GCount *cnt,
                                                                   const unsigned long long *keys) {
    extern __shared__ __align__(16) uint8_t gsm[];
    GreedySmem &S = *reinterpret_cast<GreedySmem *>(gsm);
    const GJob &G = J.j[blockIdx.x];
    GCount &C = cnt[blockIdx.x];
    const int part = C.part, cand = C.cand, maxc = G.max_corners;
    if (part > GF_TOP_MAX) {  // does not fit: straight to the second pass
        if (threadIdx.x == 0) {
            C.retry = 1;
            C.kept = 0;
            C.lo = 0;
            C.part = cand;
        }
        return;
    }
    const unsigned long long lo = C.lo;
    if (threadIdx.x == 0) S.n = 0;
    for (int c = threadIdx.x; c < G.gr_cx * G.gr_cy; c += blockDim.x) S.head[c] = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < cand; i += blockDim.x) {
        const unsigned long long k = keys[(size_t)G.px0 + i];
        if (k >= lo) S.key[atomicAdd(&S.n, 1)] = k;
    }
    __syncthreads();
    int N = 1;
    while (N < part) N <<= 1;
    for (int i = part + threadIdx.x; i < N; i += blockDim.x) S.key[i] = 0ull;
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const int p = i ^ j;
                if (p > i) {
                    const unsigned long long a = S.key[i], b = S.key[p];
                    if (((i & k) == 0) ? (a < b) : (a > b)) {
                        S.key[i] = b;
                        S.key[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < part; i += blockDim.x) {
        const unsigned p = key_pixel(S.key[i]) - (unsigned)G.px0;
        S.pxy[i] = (p % (unsigned)G.w) | ((p / (unsigned)G.w) << 16);
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int d2 = J.min_dist * J.min_dist, cs = G.gr_cell;
    int kept = 0;
    for (int base = 0; base < part && kept < maxc; base += 32) {
        const int i = base + lane;
        const bool have = i < part;
        const unsigned long long key = have ? S.key[i] : 0ull;
        const uint32_t pq = have ? S.pxy[i] : 0u;
        const int x = (int)(pq & 0xffffu), y = (int)(pq >> 16);
        bool ok = have;
        if (ok) {  // against the corners kept by earlier chunks
            const int cx = x / cs, cy = y / cs;
            for (int dy = -1; dy <= 1 && ok; ++dy) {
                const int yy = cy + dy;
                if (yy < 0 || yy >= G.gr_cy) continue;
                for (int dx = -1; dx <= 1 && ok; ++dx) {
                    const int xx = cx + dx;
                    if (xx < 0 || xx >= G.gr_cx) continue;
                    for (int e = S.head[yy * G.gr_cx + xx]; e >= 0; e = S.next[e]) {
                        const uint32_t q = S.kxy[e];
                        const int ex = (int)(q & 0xffffu) - x, ey = (int)(q >> 16) - y;
                        if (ex * ex + ey * ey < d2) {
                            ok = false;
                            break;
                        }
                    }
                }
            }
        }
        unsigned conflict = 0;  // earlier lanes of this chunk closer than min_dist
        for (int j = 0; j < 32; ++j) {
            const int xj = __shfl_sync(0xffffffffu, x, j), yj = __shfl_sync(0xffffffffu, y, j);
            const int ex = xj - x, ey = yj - y;
            if (j < lane && ex * ex + ey * ey < d2) conflict |= 1u << j;
        }
        const unsigned okm = __ballot_sync(0xffffffffu, ok);
        unsigned K = 0;
        for (int j = 0; j < 32; ++j) {
            const unsigned cj = __shfl_sync(0xffffffffu, conflict, j);
            if (((okm >> j) & 1u) && !(cj & K)) K |= 1u << j;
        }
        const int pos = kept + __popc(K & ((1u << lane) - 1u));
        if (((K >> lane) & 1u) && pos < maxc) {
            const int c = (y / cs) * G.gr_cx + (x / cs);
            S.kxy[pos] = (uint32_t)x | ((uint32_t)y << 16);
            S.next[pos] = (int16_t)atomicExch(&S.head[c], pos);
            G.out[pos] = make_float2((float)x, (float)y);
            if (G.out_score) G.out_score[pos] = __uint_as_float((unsigned)(key >> 32));
        }
        kept = min(maxc, kept + __popc(K));
        __syncwarp();
    }
    if (lane == 0) {
        const bool retry = kept < maxc && part < cand;
        C.retry = retry ? 1 : 0;
        if (retry) {
            C.kept = 0;
            C.lo = 0;
            C.part = cand;
        } else {
            *G.out_count = kept;
        }
    }
}

// Descending bitonic sort of a[0..N) (N a power of two) by one CTA.
__device__ __forceinline__ void bitonic_desc(unsigned long long *a, int N) {
    for (int k = 2; k <= N; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const int p = i ^ j;
                if (p > i) {
                    const unsigned long long x = a[i], y = a[p];
                    if (((i & k) == 0) ? (x < y) : (x > y)) {
                        a[i] = y;
                        a[p] = x;
                    }
                }
            }
            __syncthreads();
        }
}

// One CTA per frame: the first max_corners kept keys in descending order.
// Up to 2048 kept keys are sorted whole in shared memory.  Otherwise the
// smallest set of top histogram bins (12 score bits: exponent and three
// mantissa bits) that holds max_corners keys -- exactly the keys greater than
// or equal to its lowest bin's lower bound -- is sorted there if it fits,
// else the whole kept set is sorted in global memory (its segment is a power
// of two long).
__global__ void __launch_bounds__(GF_OUT_THREADS) k_gftt_output(const __grid_constant__ GJobs J, const GCount *cnt,
                                                                unsigned long long *kept) {
    extern __shared__ __align__(16) unsigned long long sk[];
    __shared__ int hist[GF_HIST];
    __shared__ int s_bin, s_n;
    const GJob &G = J.j[blockIdx.x];
    if (!cnt[blockIdx.x].retry) return;  // the first pass already wrote this frame's corners
    unsigned long long *seg = kept + G.kept0;
    const int K = cnt[blockIdx.x].kept;
    const int m = min(K, G.max_corners);
    unsigned long long *a = sk;
    int N = 1;
    if (K <= 2048) {  // small: sort everything
        while (N < K) N <<= 1;
        for (int i = threadIdx.x; i < N; i += blockDim.x) sk[i] = i < K ? seg[i] : 0ull;
        __syncthreads();
    } else {
        for (int i = threadIdx.x; i < GF_HIST; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += blockDim.x) atomicAdd(&hist[(int)(seg[i] >> 52)], 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0, b = GF_HIST - 1;
            for (; b > 0; --b) {
                acc += hist[b];
                if (acc >= m) break;
            }
            if (b == 0) acc += hist[0];
            s_bin = b;
            s_n = acc;
        }
        __syncthreads();
        const int nsel = s_n;
        __syncthreads();
        if (nsel <= GF_SMEM_SORT) {
            if (threadIdx.x == 0) s_n = 0;
            __syncthreads();
            const unsigned long long lo = (unsigned long long)s_bin << 52;
            for (int i = threadIdx.x; i < K; i += blockDim.x) {
                const unsigned long long k = seg[i];
                if (k >= lo) sk[atomicAdd(&s_n, 1)] = k;
            }
            __syncthreads();
            while (N < nsel) N <<= 1;
            for (int i = nsel + threadIdx.x; i < N; i += blockDim.x) sk[i] = 0ull;
            __syncthreads();
        } else {
            while (N < K) N <<= 1;
            for (int i = K + threadIdx.x; i < N && i < G.kept_cap; i += blockDim.x) seg[i] = 0ull;
            __syncthreads();
            a = seg;
        }
    }
    bitonic_desc(a, N);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const unsigned long long k = a[i];
        const unsigned p = key_pixel(k) - (unsigned)G.px0;
        G.out[i] = make_float2((float)(p % (unsigned)G.w), (float)(p / (unsigned)G.w));
        if (G.out_score) G.out_score[i] = __uint_as_float((unsigned)(k >> 32));
    }
    if (threadIdx.x == 0) *G.out_count = m;
}

}  // namespace vt

using namespace vt;

struct vt_gftt {
    long long cap;  // pixels of all frames of one call
    GCount *cnt;  // [kMaxGfttJobs]
    int *und;     // [3] undecided candidates per round
    unsigned long long *keys, *skeys, *kept;
    int *rank, *cell_count, *cell_start, *hist;
    uint8_t *state;
    int max_w, max_h;
    int sms, select_grid;
};

static long long pow2_at_least(long long v) {
    long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

extern "C" {

vt_status vt_gftt_create_pixels(long long max_pixels, vt_gftt **out) {
    if (!out || max_pixels <= 0 || max_pixels > (1ll << 31) - 1) return VT_ERR_ARG;
    vt_gftt *g = (vt_gftt *)calloc(1, sizeof(vt_gftt));
    if (!g) return VT_ERR_OOM;
    g->cap = max_pixels;
    g->max_w = g->max_h = 65535;
    const size_t px = (size_t)max_pixels;
    // cells: at most one per pixel plus one end entry per frame
    bool ok = cudaMalloc(&g->cnt, sizeof(GCount) * kMaxGfttJobs) == cudaSuccess &&
              cudaMalloc(&g->und, 4 * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&g->keys, sizeof(unsigned long long) * px) == cudaSuccess &&
              cudaMalloc(&g->skeys, sizeof(unsigned long long) * px) == cudaSuccess &&
              cudaMalloc(&g->kept, sizeof(unsigned long long) * 2 * px) == cudaSuccess &&
              cudaMalloc(&g->rank, sizeof(int) * px) == cudaSuccess && cudaMalloc(&g->state, px) == cudaSuccess &&
              cudaMalloc(&g->cell_count, sizeof(int) * (px + kMaxGfttJobs)) == cudaSuccess &&
              cudaMalloc(&g->cell_start, sizeof(int) * (px + kMaxGfttJobs)) == cudaSuccess &&
              cudaMalloc(&g->hist, sizeof(int) * GF_HIST * kMaxGfttJobs) == cudaSuccess;
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

vt_status vt_gftt_create(int max_w, int max_h, vt_gftt **out) {
    if (!out || max_w <= 0 || max_h <= 0 || max_w > 65535 || max_h > 65535) return VT_ERR_ARG;
    const vt_status st = vt_gftt_create_pixels((long long)max_w * max_h, out);
    if (st == VT_OK) {
        (*out)->max_w = max_w;
        (*out)->max_h = max_h;
    }
    return st;
}

void vt_gftt_free(vt_gftt *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    cudaFree(g->cnt);
    cudaFree(g->und);
    cudaFree(g->keys);
    cudaFree(g->skeys);
    cudaFree(g->kept);
    cudaFree(g->rank);
    cudaFree(g->state);
    cudaFree(g->cell_count);
    cudaFree(g->cell_start);
    cudaFree(g->hist);
    free(g);
}

vt_status vt_gftt_detect_many(vt_gftt *g, const vt_gftt_job *jobs, int njobs, const vt_gftt_params *prm,
                              void *cuda_stream) {
    if (!g || !prm || njobs < 0 || njobs > kMaxGfttJobs || (njobs > 0 && !jobs)) return VT_ERR_ARG;
    if (!(prm->quality >= 0.f) || prm->min_dist < 1 || prm->nms_radius < 0 || prm->nms_radius > GF_MAX_NMS ||
        prm->block_radius < 0 || prm->block_radius > GF_MAX_BR || prm->border < 0)
        return VT_ERR_ARG;
    GJobs J;
    J.n = njobs;
    J.br = prm->block_radius;
    J.nms = prm->nms_radius;
    J.border = prm->border;
    J.min_dist = prm->min_dist;
    J.quality = prm->quality;
    long long px = 0, kept = 0;
    int tiles = 0, cells = 0;
    for (int i = 0; i < njobs; ++i) {
        const vt_gftt_job &jb = jobs[i];
        if (!jb.pyr || jb.level < 0 || jb.level >= jb.pyr->levels || jb.pyr->gtype != VT_GRAD_S16 ||
            !jb.corners_out || !jb.count_out || jb.max_corners < 0 || jb.max_corners > GF_MAX_CORNERS ||
            jb.n_mask < 0 || (jb.n_mask > 0 && !jb.mask_pts))
            return VT_ERR_ARG;
        const Level &L = jb.pyr->lv[jb.level];
        if (L.w > g->max_w || L.h > g->max_h) return VT_ERR_ARG;
        GJob &G = J.j[i];
        G.grad = L.grad;
        G.gpitch = L.gpitch;
        G.w = L.w;
        G.h = L.h;
        G.tiles_x = (L.w + GF_TX - 1) / GF_TX;
        G.tile0 = tiles;
        tiles += G.tiles_x * ((L.h + GF_TY - 1) / GF_TY);
        G.px0 = (int)px;
        px += (long long)L.w * L.h;
        G.cells_x = (L.w + prm->min_dist - 1) / prm->min_dist;
        G.cells_y = (L.h + prm->min_dist - 1) / prm->min_dist;
        G.cell0 = cells;
        cells += G.cells_x * G.cells_y + 1;
        G.kept_cap = (int)pow2_at_least((long long)L.w * L.h);
        G.kept0 = kept;
        kept += G.kept_cap;
        G.mask = reinterpret_cast<const float2 *>(jb.mask_pts);
        G.n_mask = jb.n_mask;
        G.out = reinterpret_cast<float2 *>(jb.corners_out);
        G.out_score = jb.scores_out;
        G.out_count = jb.count_out;
        G.max_corners = jb.max_corners;
        G.gr_cell = prm->min_dist;
        while ((long long)((L.w + G.gr_cell - 1) / G.gr_cell) * ((L.h + G.gr_cell - 1) / G.gr_cell) > GF_GR_CELLS)
            ++G.gr_cell;
        G.gr_cx = (L.w + G.gr_cell - 1) / G.gr_cell;
        G.gr_cy = (L.h + G.gr_cell - 1) / G.gr_cell;
        if (px > g->cap) return VT_ERR_ARG;
    }
    if (kept > 2 * g->cap) return VT_ERR_ARG;
    J.tiles = tiles;
    if (njobs == 0) return VT_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(g->cnt, 0, sizeof(GCount) * njobs, s) != cudaSuccess ||
        cudaMemsetAsync(g->und, 0, 4 * sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(g->cell_count, 0, sizeof(int) * (size_t)cells, s) != cudaSuccess ||
        cudaMemsetAsync(g->hist, 0, sizeof(int) * GF_HIST * (size_t)njobs, s) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    static const bool attr = [] {  // once, thread-safe static initialisation
        return cudaFuncSetAttribute(k_gftt_output, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(GF_SMEM_SORT * sizeof(unsigned long long))) == cudaSuccess &&
               cudaFuncSetAttribute(k_gftt_greedy_top, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(GreedySmem)) == cudaSuccess;
    }();
    (void)attr;
    const dim3 blk(GF_TX, GF_TY);
    int max_mask = 0;
    for (int i = 0; i < njobs; ++i) max_mask = max(max_mask, jobs[i].n_mask);
    if (max_mask > 0) {  // the state bytes serve as the mask map until the cell scatter rewrites them
        if (cudaMemsetAsync(g->state, 0, (size_t)px, s) != cudaSuccess) {
            cudaGetLastError();
            return VT_ERR_CUDA;
        }
        const dim3 mgrid((unsigned)min(1024, (max_mask + 7) / 8), (unsigned)njobs);
        k_gftt_mask<<<mgrid, 256, 0, s>>>(J, g->state);
    }
    switch (prm->block_radius) {
        case 0: k_gftt_local<0><<<tiles, blk, 0, s>>>(J, g->cnt, g->state, g->skeys); break;
        case 1: k_gftt_local<1><<<tiles, blk, 0, s>>>(J, g->cnt, g->state, g->skeys); break;
        case 2: k_gftt_local<2><<<tiles, blk, 0, s>>>(J, g->cnt, g->state, g->skeys); break;
        default: k_gftt_local<3><<<tiles, blk, 0, s>>>(J, g->cnt, g->state, g->skeys); break;
    }
    const dim3 cgrid((unsigned)((4 * g->sms + njobs - 1) / njobs), (unsigned)njobs);
    k_gftt_filter<<<cgrid, GF_GRID_THREADS, 0, s>>>(J, g->cnt, g->skeys, g->keys);
    k_gftt_hist<<<cgrid, GF_GRID_THREADS, 0, s>>>(J, g->cnt, g->keys, g->hist);
    k_gftt_top<<<njobs, GF_HIST / 4, 0, s>>>(J, g->cnt, g->hist);
    k_gftt_greedy_top<<<njobs, GF_GR_THREADS, sizeof(GreedySmem), s>>>(J, g->cnt, g->keys);
    {  // second pass, for the frames the first could not settle (no-ops for the others)
        const int pass = 2;
        k_gftt_cell_count<<<cgrid, GF_GRID_THREADS, 0, s>>>(J, g->cnt, g->keys, g->cell_count, g->rank, pass);
        k_gftt_cell_scan<<<njobs, GF_SCAN_THREADS, 0, s>>>(J, g->cnt, g->cell_count, g->cell_start, pass);
        k_gftt_cell_scatter<<<cgrid, GF_GRID_THREADS, 0, s>>>(J, g->cnt, g->keys, g->cell_start, g->rank, g->skeys,
                                                              g->state, pass);
        GCount *cnt = g->cnt;
        const unsigned long long *skeys = g->skeys;
        const int *cell_start = g->cell_start;
        uint8_t *state = g->state;
        int *und = g->und;
        unsigned long long *keptp = g->kept;
        int pass_arg = pass;
        void *args[] = {(void *)&J,     (void *)&cnt, (void *)&skeys, (void *)&cell_start,
                        (void *)&state, (void *)&und, (void *)&keptp, (void *)&pass_arg};
        if (cudaLaunchCooperativeKernel((const void *)k_gftt_select, g->select_grid, GF_MIS_THREADS, args, 0, s) !=
            cudaSuccess) {
            cudaGetLastError();
            return VT_ERR_CUDA;
        }
    }
    k_gftt_output<<<njobs, GF_OUT_THREADS, GF_SMEM_SORT * sizeof(unsigned long long), s>>>(J, g->cnt, g->kept);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

vt_status vt_gftt_detect(vt_gftt *g, const vt_pyramid *p, int level, const vt_gftt_params *prm, const float *mask_pts,
                         int n_mask, float *corners_out, float *scores_out, int *count_out, void *cuda_stream) {
    if (!g || !p || !prm || !corners_out || !count_out) return VT_ERR_ARG;
    vt_gftt_job jb;
    jb.pyr = p;
    jb.level = level;
    jb.mask_pts = mask_pts;
    jb.n_mask = n_mask;
    jb.corners_out = corners_out;
    jb.scores_out = scores_out;
    jb.count_out = count_out;
    jb.max_corners = prm->max_corners;
    return vt_gftt_detect_many(g, &jb, 1, prm, cuda_stream);
}

}  // extern "C"
