// Track bookkeeping (K8) for many camera streams at once: identity
// carry-over with age-priority thinning, and spawning of new tracks from
// detections up to each stream's cap.  One CTA per stream; every stream's
// pool stays on the device, counts included, so a step needs no host round
// trip.
//
//   k_tracks_carry  survivors of the temporal step (status 1) in index order,
//                   ages + 1, sorted by (age desc, index asc) in shared
//                   memory; the greedy min-distance thinning in that order is
//                   resolved in parallel rounds over a cell grid in shared
//                   memory (a survivor is kept when no kept higher-priority
//                   survivor lies closer than min_dist, dropped when one
//                   does); kept survivors rewrite the pool in priority order
//                   and, optionally, a detector mask padded with NaN.
//   k_tracks_spawn  accepted detections, in their priority order, appended
//                   until the pool holds `cap` features, with identities
//                   next_id, next_id + 1, ... and age 1.
// Distances are single precision, dx*dx + dy*dy rounded operation by
// operation, as in the oracle, so the result is exact.
#include <cmath>
#include <cstdint>

#include "vt_internal.cuh"

namespace vt {

constexpr int TK_THREADS = 1024;
constexpr int TK_PER = VT_POOL_MAX / TK_THREADS;  // pool entries per thread
constexpr int TK_MAX_CELLS = 4096;
constexpr int kMaxPoolJobs = 192;
enum : uint8_t { TK_UNDECIDED = 0, TK_KEPT = 1, TK_DROPPED = 2 };

struct CarryJobs {
    int n;
    float min_dist;
    vt_carry_job j[kMaxPoolJobs];
};

struct SpawnJobs {
    int n;
    vt_spawn_job j[kMaxPoolJobs];
};

// Exclusive block-wide scan of one int per thread (TK_THREADS threads);
// returns the total through *total.
__device__ __forceinline__ int block_scan(int v, int *warp_sums, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;  // inclusive sums of the warps
    }
    __syncthreads();
    const int excl = x - v + (wid > 0 ? warp_sums[wid - 1] : 0);
    if (total) *total = warp_sums[31];
    __syncthreads();
    return excl;
}

__device__ __forceinline__ float dist2(float2 a, float2 b) {
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

struct CarrySmem {
    unsigned long long key[VT_POOL_MAX];  // (age << 32) | ~rank, sorted descending
    float2 pos[VT_POOL_MAX];              // survivor positions by survivor rank
    int32_t id[VT_POOL_MAX];
    int32_t age[VT_POOL_MAX];  // already + 1
    int16_t cell_of[VT_POOL_MAX];          // by priority position
    int16_t member[VT_POOL_MAX];           // priority positions grouped by cell
    int cell_start[TK_MAX_CELLS + 1];
    int cursor[TK_MAX_CELLS];
    uint8_t state[VT_POOL_MAX];            // by priority position
    int warp_sums[32];
    float red[4][32];
};

__global__ void __launch_bounds__(TK_THREADS) k_tracks_carry(const __grid_constant__ CarryJobs J) {
    extern __shared__ __align__(16) uint8_t tk_smem[];
    CarrySmem &S = *reinterpret_cast<CarrySmem *>(tk_smem);
    const vt_carry_job &jb = J.j[blockIdx.x];
    const vt_track_pool &P = jb.pool;
    const int n = min(*P.count, P.cap);
    const float2 *tracked = reinterpret_cast<const float2 *>(jb.tracked);
    const int t = threadIdx.x;
    // 1. survivors in index order (TK_PER consecutive entries per thread)
    int mine = 0;
#pragma unroll
    for (int k = 0; k < TK_PER; ++k) {
        const int i = t * TK_PER + k;
        mine += (i < n && jb.status[i] != 0) ? 1 : 0;
    }
    int m;
    int r = block_scan(mine, S.warp_sums, &m);
#pragma unroll
    for (int k = 0; k < TK_PER; ++k) {
        const int i = t * TK_PER + k;
        if (i < n && jb.status[i] != 0) {
            S.pos[r] = tracked[i];
            S.id[r] = P.ids[i];
            S.age[r] = P.ages[i] + 1;
            ++r;
        }
    }
    __syncthreads();
    // 2. priority order: age descending, then survivor rank ascending (bitonic, descending keys)
    int N = 1;
    while (N < m) N <<= 1;
    for (int i = t; i < N; i += TK_THREADS)
        S.key[i] = i < m ? ((unsigned long long)(uint32_t)S.age[i] << 32) | (0xffffffffu - (unsigned)i) : 0ull;
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = t; i < N; i += TK_THREADS) {
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
    // 3. cell grid over the survivors' bounding box: cells wider than
    //    min_dist (by 0.1 %, so rounding cannot separate a close pair by two
    //    cells), at most TK_MAX_CELLS of them
    float lo_x = INFINITY, lo_y = INFINITY, hi_x = -INFINITY, hi_y = -INFINITY;
    for (int i = t; i < m; i += TK_THREADS) {
        const float2 p = S.pos[i];
        if (!isfinite(p.x) || !isfinite(p.y)) continue;  // non-finite points share cell 0
        lo_x = fminf(lo_x, p.x);
        lo_y = fminf(lo_y, p.y);
        hi_x = fmaxf(hi_x, p.x);
        hi_y = fmaxf(hi_y, p.y);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        lo_x = fminf(lo_x, __shfl_xor_sync(0xffffffffu, lo_x, o));
        lo_y = fminf(lo_y, __shfl_xor_sync(0xffffffffu, lo_y, o));
        hi_x = fmaxf(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, o));
        hi_y = fmaxf(hi_y, __shfl_xor_sync(0xffffffffu, hi_y, o));
    }
    if ((t & 31) == 0) {
        S.red[0][t >> 5] = lo_x;
        S.red[1][t >> 5] = lo_y;
        S.red[2][t >> 5] = hi_x;
        S.red[3][t >> 5] = hi_y;
    }
    __syncthreads();
    lo_x = S.red[0][0], lo_y = S.red[1][0], hi_x = S.red[2][0], hi_y = S.red[3][0];
    for (int w = 1; w < 32; ++w) {
        lo_x = fminf(lo_x, S.red[0][w]);
        lo_y = fminf(lo_y, S.red[1][w]);
        hi_x = fmaxf(hi_x, S.red[2][w]);
        hi_y = fmaxf(hi_y, S.red[3][w]);
    }
    const float md = J.min_dist, md2 = __fmul_rn(md, md);
    float cs = md * 1.001f;
    int cx = 1, cy = 1;
    if (lo_x <= hi_x && lo_y <= hi_y) {  // some finite survivor
        int tries = 0;
        for (;; ++tries) {
            const float fx = floorf((hi_x - lo_x) / cs) + 1.f, fy = floorf((hi_y - lo_y) / cs) + 1.f;
            if (fx * fy <= (float)TK_MAX_CELLS) {
                cx = (int)fx;
                cy = (int)fy;
                break;
            }
            if (tries == 64) break;  // one cell for everything: still exact, only slower
            cs *= 1.5f;
        }
    } else {
        lo_x = lo_y = 0.f;
    }
    for (int c = t; c < TK_MAX_CELLS; c += TK_THREADS) S.cursor[c] = 0;
    __syncthreads();
    for (int q = t; q < m; q += TK_THREADS) {  // q: priority position
        const float2 p = S.pos[0xffffffffu - (unsigned)(S.key[q] & 0xffffffffu)];
        const int ix = clampi((int)floorf((p.x - lo_x) / cs), 0, cx - 1);
        const int iy = clampi((int)floorf((p.y - lo_y) / cs), 0, cy - 1);
        const int c = ix + cx * iy;
        S.cell_of[q] = (int16_t)c;
        atomicAdd(&S.cursor[c], 1);
        S.state[q] = TK_UNDECIDED;
    }
    __syncthreads();
    {  // cell starts: exclusive scan of the counts (TK_MAX_CELLS / TK_THREADS cells per thread)
        constexpr int CPT = TK_MAX_CELLS / TK_THREADS;
        int cnt[CPT], sum = 0;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            cnt[k] = S.cursor[t * CPT + k];
            sum += cnt[k];
        }
        int run = block_scan(sum, S.warp_sums, nullptr);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            S.cell_start[t * CPT + k] = run;
            S.cursor[t * CPT + k] = run;
            run += cnt[k];
        }
        if (t == TK_THREADS - 1) S.cell_start[TK_MAX_CELLS] = run;
    }
    __syncthreads();
    // members of each cell (order within a cell does not matter)
    for (int q = t; q < m; q += TK_THREADS) S.member[atomicAdd(&S.cursor[S.cell_of[q]], 1)] = (int16_t)q;
    __syncthreads();
    // 4. greedy thinning in parallel rounds
    for (;;) {
        int undecided = 0;
        for (int q = t; q < m; q += TK_THREADS) {
            if (S.state[q] != TK_UNDECIDED) continue;
            const float2 p = S.pos[0xffffffffu - (unsigned)(S.key[q] & 0xffffffffu)];
            const int c = S.cell_of[q], ccx = c % cx, ccy = c / cx;
            bool blocked = false, dropped = false;
            for (int dy = -1; dy <= 1 && !dropped; ++dy) {
                const int yy = ccy + dy;
                if (yy < 0 || yy >= cy) continue;
                for (int dx = -1; dx <= 1 && !dropped; ++dx) {
                    const int xx = ccx + dx;
                    if (xx < 0 || xx >= cx) continue;
                    const int cc = yy * cx + xx;
                    for (int e = S.cell_start[cc]; e < S.cell_start[cc + 1]; ++e) {
                        const int o = S.member[e];
                        if (o >= q) continue;  // lower priority (or itself)
                        const float2 po = S.pos[0xffffffffu - (unsigned)(S.key[o] & 0xffffffffu)];
                        if (!(dist2(p, po) < md2)) continue;
                        const uint8_t so = *reinterpret_cast<volatile uint8_t *>(&S.state[o]);
                        if (so == TK_KEPT) {
                            dropped = true;
                            break;
                        }
                        if (so == TK_UNDECIDED) blocked = true;
                    }
                }
            }
            if (dropped) S.state[q] = TK_DROPPED;
            else if (!blocked) S.state[q] = TK_KEPT;
            else undecided = 1;
        }
        if (!__syncthreads_or(undecided)) break;
    }
    // 5. the kept survivors, in priority order, rewrite the pool
    int kept_mine = 0;
#pragma unroll
    for (int k = 0; k < TK_PER; ++k) {
        const int q = t * TK_PER + k;
        kept_mine += (q < m && S.state[q] == TK_KEPT) ? 1 : 0;
    }
    int kept;
    int w = block_scan(kept_mine, S.warp_sums, &kept);
    float2 *pts = reinterpret_cast<float2 *>(P.pts);
    float2 *mask = reinterpret_cast<float2 *>(jb.mask);
#pragma unroll
    for (int k = 0; k < TK_PER; ++k) {
        const int q = t * TK_PER + k;
        if (q < m && S.state[q] == TK_KEPT) {
            const int s = 0xffffffffu - (unsigned)(S.key[q] & 0xffffffffu);
            pts[w] = S.pos[s];
            P.ids[w] = S.id[s];
            P.ages[w] = S.age[s];
            if (mask) mask[w] = S.pos[s];
            ++w;
        }
    }
    if (mask)
        for (int i = kept + t; i < P.cap; i += TK_THREADS) mask[i] = make_float2(NAN, NAN);
    if (t == 0) *P.count = kept;
}

__global__ void __launch_bounds__(TK_THREADS) k_tracks_spawn(const __grid_constant__ SpawnJobs J) {
    __shared__ int warp_sums[32];
    const vt_spawn_job &jb = J.j[blockIdx.x];
    const vt_track_pool &P = jb.pool;
    const int c0 = min(*P.count, P.cap), nc = *jb.n_corners;
    const int room = P.cap - c0, id0 = *P.next_id;
    const float2 *corners = reinterpret_cast<const float2 *>(jb.corners);
    float2 *pts = reinterpret_cast<float2 *>(P.pts);
    int base = 0;
    for (int b0 = 0; b0 < nc && base < room; b0 += TK_THREADS) {  // chunks of TK_THREADS detections, in order
        const int i = b0 + threadIdx.x;
        const int a = (i < nc && (!jb.accept || jb.accept[i] != 0)) ? 1 : 0;
        int total;
        const int r = base + block_scan(a, warp_sums, &total);
        if (a && r < room) {
            pts[c0 + r] = corners[i];
            P.ids[c0 + r] = id0 + r;
            P.ages[c0 + r] = 1;
        }
        base += total;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int added = min(base, room);
        *P.count = c0 + added;
        *P.next_id = id0 + added;
    }
}

static bool pool_ok(const vt_track_pool &p) {
    return p.pts && p.ids && p.ages && p.count && p.next_id && p.cap >= 1 && p.cap <= VT_POOL_MAX;
}

}  // namespace vt

using namespace vt;

extern "C" {

vt_status vt_tracks_carry(const vt_carry_job *jobs, int njobs, float min_dist, void *cuda_stream) {
    if (njobs < 0 || njobs > kMaxPoolJobs || (njobs > 0 && !jobs) || !(min_dist > 0.f) || !std::isfinite(min_dist))
        return VT_ERR_ARG;
    for (int i = 0; i < njobs; ++i)
        if (!pool_ok(jobs[i].pool) || !jobs[i].tracked || !jobs[i].status) return VT_ERR_ARG;
    if (njobs == 0) return VT_OK;
    CarryJobs J;  // copied into the launch's parameters
    J.n = njobs;
    J.min_dist = min_dist;
    for (int i = 0; i < njobs; ++i) J.j[i] = jobs[i];
    static const bool attr = [] {  // once, thread-safe static initialisation
        return cudaFuncSetAttribute(k_tracks_carry, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(CarrySmem)) == cudaSuccess;
    }();
    (void)attr;
    k_tracks_carry<<<njobs, TK_THREADS, sizeof(CarrySmem), (cudaStream_t)cuda_stream>>>(J);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

vt_status vt_tracks_spawn(const vt_spawn_job *jobs, int njobs, void *cuda_stream) {
    if (njobs < 0 || njobs > kMaxPoolJobs || (njobs > 0 && !jobs)) return VT_ERR_ARG;
    for (int i = 0; i < njobs; ++i)
        if (!pool_ok(jobs[i].pool) || !jobs[i].corners || !jobs[i].n_corners) return VT_ERR_ARG;
    if (njobs == 0) return VT_OK;
    SpawnJobs J;
    J.n = njobs;
    for (int i = 0; i < njobs; ++i) J.j[i] = jobs[i];
    k_tracks_spawn<<<njobs, TK_THREADS, 0, (cudaStream_t)cuda_stream>>>(J);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

}  // extern "C"
