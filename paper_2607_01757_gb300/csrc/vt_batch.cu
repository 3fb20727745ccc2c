// Batched tracking (K5): many frames and tracking tasks of independent camera
// streams in a fixed sequence of persistent launches.
//
//   H2D   job tables (pinned staging -> device, one copy)
//   K1+K2 per pyramid level: one persistent launch over the tiles of every
//         frame that has that level (level 0 also copies the caller image)
//   K2    Scharr of each frame's last level
//   K3    one persistent KLT launch: warps take points from a device work
//         counter (one atomicAdd per point) across all tasks
//   K7    (when gate tasks are set) the stereo triangulation gate over every
//         gate task's pairs, one thread per pair
//
// Grid sizes do not depend on the batch (SMs x resident CTAs), so one CUDA
// graph per topology (deepest pyramid, gradient type, window) replays any
// batch: the host only rewrites the pinned tables between replays.  Two
// staging buffers let the host prepare run t+1 while run t executes.
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "vt_klt.cuh"

namespace vt {

template <int WIN, int GT, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, KltOcc<WIN>::min_blocks * 4 / WARPS)
    k_klt_batch(const uint8_t *tab, int *counter) {
    extern __shared__ __align__(16) uint8_t klt_smem[];
    KSmem<WIN> &sm = reinterpret_cast<KSmem<WIN> *>(klt_smem)[threadIdx.x >> 5];
    ksmem_init<WIN>(sm, threadIdx.x & 31);
    const BatchHdr *H = reinterpret_cast<const BatchHdr *>(tab);
    const BTask *tasks = reinterpret_cast<const BTask *>(tab + H->off_tasks);
    const int *p0s = reinterpret_cast<const int *>(tab + H->off_prefix);
    const int total = H->total_points, nt = H->ntasks;
    const KParams P = H->P;
    const int lane = threadIdx.x & 31;
    pdl_wait();  // the pyramids are the previous launch's output
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(counter, 1);
        p = __shfl_sync(kFull, p, 0);
        if (p >= total) break;
        int lo = 0, hi = nt - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(p0s + mid) <= p) lo = mid;
            else hi = mid - 1;
        }
        const BTask &t = tasks[lo];
        const int i = p - t.p0;
        if (t.n_dev && i >= __ldg(t.n_dev)) continue;  // beyond the device-side count
        const float2 u = t.pts_in[i];
        KParams Pt = P;
        Pt.levels = t.levels;
        KOut o;
        track_point_dir<WIN, GT, false>(t.I, t.J, Pt, u.x, u.y, t.fb != 0, false, 0.f, 0.f, lane, sm, o);
        if (lane == 0) {
            if (o.reason == kReasonPending) {  // left to k_klt_batch_f64
                t.status[i] = kStatusPending;
                continue;
            }
            t.pts_out[i] = make_float2(o.x, o.y);
            t.status[i] = (uint8_t)o.status;
            if (t.err) t.err[i] = o.status ? o.err : 0.f;
            if (t.reason) t.reason[i] = (uint8_t)o.reason;
            if (t.flops) t.flops[i] = klt_flops(WIN, o);
        }
    }
}

// The FP64-capable pass of a batched run (launched only when an accepted
// template can be ill-conditioned, fp64_needed): warps stride over every
// point of the run and track again, with ill-conditioned levels in FP64,
// those the FP32 launch left pending.
template <int WIN, int GT>
__global__ void __launch_bounds__(128) k_klt_batch_f64(const uint8_t *tab) {
    extern __shared__ __align__(16) uint8_t klt_smem[];
    KSmem<WIN> &sm = reinterpret_cast<KSmem<WIN> *>(klt_smem)[threadIdx.x >> 5];
    ksmem_init<WIN>(sm, threadIdx.x & 31);
    const BatchHdr *H = reinterpret_cast<const BatchHdr *>(tab);
    const BTask *tasks = reinterpret_cast<const BTask *>(tab + H->off_tasks);
    const int *p0s = reinterpret_cast<const int *>(tab + H->off_prefix);
    const int total = H->total_points, nt = H->ntasks;
    const KParams P = H->P;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < total; p += nwarps) {
        int lo = 0, hi = nt - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(p0s + mid) <= p) lo = mid;
            else hi = mid - 1;
        }
        const BTask &t = tasks[lo];
        const int i = p - t.p0;
        if (t.n_dev && i >= __ldg(t.n_dev)) continue;
        if (t.status[i] != kStatusPending) continue;
        const float2 u = t.pts_in[i];
        KParams Pt = P;
        Pt.levels = t.levels;
        KOut o;
        track_point_dir<WIN, GT, true>(t.I, t.J, Pt, u.x, u.y, t.fb != 0, false, 0.f, 0.f, lane, sm, o);
        if (lane == 0) {
            t.pts_out[i] = make_float2(o.x, o.y);
            t.status[i] = (uint8_t)o.status;
            if (t.err) t.err[i] = o.status ? o.err : 0.f;
            if (t.reason) t.reason[i] = (uint8_t)o.reason;
            if (t.flops) t.flops[i] = klt_flops(WIN, o);
        }
    }
}

template <int WIN, int GT>
static void launch_f64_win(const uint8_t *tab, int grid, cudaStream_t s) {
    const size_t smem = 4 * sizeof(KSmem<WIN>);
    static const bool attr = [smem] {  // once, thread-safe static initialisation
        return cudaFuncSetAttribute(k_klt_batch_f64<WIN, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem) == cudaSuccess;
    }();
    (void)attr;
    k_klt_batch_f64<WIN, GT><<<grid, 128, smem, s>>>(tab);
}

template <int GT>
static void launch_f64_gt(const uint8_t *tab, int win, int grid, cudaStream_t s) {
    switch (win) {
        case 9: launch_f64_win<9, GT>(tab, grid, s); break;
        case 15: launch_f64_win<15, GT>(tab, grid, s); break;
        case 21: launch_f64_win<21, GT>(tab, grid, s); break;
        case 31: launch_f64_win<31, GT>(tab, grid, s); break;
    }
}

// The FP64-capable pass over the run's pending points (stream-ordered after
// the FP32 tracking launch).
static vt_status launch_klt_f64(const uint8_t *tab, int win, int gtype, int grid, cudaStream_t s) {
    if (gtype == VT_GRAD_F16)
        launch_f64_gt<VT_GRAD_F16>(tab, win, grid, s);
    else if (gtype == VT_GRAD_NONE)
        launch_f64_gt<VT_GRAD_NONE>(tab, win, grid, s);
    else
        launch_f64_gt<VT_GRAD_S16>(tab, win, grid, s);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

typedef void (*KltBatchFn)(const uint8_t *, int *);

struct KltBatchKernel {
    KltBatchFn fn;
    size_t smem;  // dynamic shared memory per CTA
};

template <int WIN, int GT, int WARPS>
static KltBatchKernel klt_batch_entry() {
    const size_t smem = WARPS * sizeof(KSmem<WIN>);
    // opt in to more than 48 KB where needed (once, thread-safe static initialisation)
    static const bool attr = [smem] {
        return cudaFuncSetAttribute(k_klt_batch<WIN, GT, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem) == cudaSuccess;
    }();
    (void)attr;
    return {k_klt_batch<WIN, GT, WARPS>, smem};
}

template <int GT, int WARPS>
static KltBatchKernel klt_batch_fn(int win) {
    switch (win) {
        case 9: return klt_batch_entry<9, GT, WARPS>();
        case 15: return klt_batch_entry<15, GT, WARPS>();
        case 21: return klt_batch_entry<21, GT, WARPS>();
        case 31: return klt_batch_entry<31, GT, WARPS>();
    }
    return {nullptr, 0};
}

static KltBatchKernel klt_batch_kernel(int win, int gtype, int warps) {
    if (gtype == VT_GRAD_F16) return warps == 8 ? klt_batch_fn<VT_GRAD_F16, 8>(win) : klt_batch_fn<VT_GRAD_F16, 4>(win);
    if (gtype == VT_GRAD_NONE)
        return warps == 8 ? klt_batch_fn<VT_GRAD_NONE, 8>(win) : klt_batch_fn<VT_GRAD_NONE, 4>(win);
    return warps == 8 ? klt_batch_fn<VT_GRAD_S16, 8>(win) : klt_batch_fn<VT_GRAD_S16, 4>(win);
}

constexpr int kGraphsPerBuffer = 8;

struct Topo {
    int maxL, gtype, win, klt_warps, klt_grid, pyr_grid, gate, fp64;
    bool operator==(const Topo &o) const {
        return maxL == o.maxL && gtype == o.gtype && win == o.win && klt_warps == o.klt_warps &&
               klt_grid == o.klt_grid && pyr_grid == o.pyr_grid && gate == o.gate && fp64 == o.fp64;
    }
};

}  // namespace vt

using namespace vt;

struct vt_batch {
    int cap_frames, cap_tasks;
    size_t tab_bytes;
    uint8_t *host[2];
    uint8_t *dev[2];
    int *counter;  // [2]
    cudaEvent_t ev[2];
    bool ev_used[2];
    int next;    // buffer the next vt_batch_set writes
    int staged;  // buffer with the latest staged tables, -1 if none
    bool fresh;  // the staged tables have not been enqueued yet (gates may still be set)
    Topo topo[2];
    // instantiated graphs per staging buffer, one per topology seen (runs of
    // different stream mixes alternate topologies, e.g. a request loop's
    // batches), replaced round robin when full
    cudaGraphExec_t exec[2][kGraphsPerBuffer];
    Topo exec_topo[2][kGraphsPerBuffer];
    int exec_next[2];
    cudaStream_t cap;
    int sms;
    int klt_warps;        // warps per CTA of the KLT launch (4 or 8)
    int klt_ctas_per_sm;  // 0 = occupancy limit
    int pyr_grid;
    int tail_grid;  // CTAs of the tail launch (one frame each at a time)
    int gate_grid;  // CTAs of the stereo-gate launch
};

namespace vt {

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static void layout(int F, int T, int &off_frames, int &off_jobs, int &off_tsrc, int &off_tasks, int &off_prefix,
                   int &off_gates, int &off_gprefix, size_t &bytes) {
    size_t o = align_up(sizeof(BatchHdr), 64);
    off_frames = (int)o;
    o = align_up(o + sizeof(BFrame) * F, 64);
    off_jobs = (int)o;
    // VT_MAX_LEVELS - 1 tiled lists of F jobs, then the tail list of up to 8 bands per frame
    o = align_up(o + sizeof(BLvlJob) * (size_t)F * (VT_MAX_LEVELS - 1 + 8), 64);
    off_tsrc = (int)o;
    o = align_up(o + sizeof(BTileSrc) * (size_t)F * (VT_MAX_LEVELS - 1), 64);
    off_tasks = (int)o;
    o = align_up(o + sizeof(BTask) * T, 64);
    off_prefix = (int)o;
    o = align_up(o + sizeof(int) * T, 64);
    off_gates = (int)o;
    o = align_up(o + sizeof(GTask) * T, 64);
    off_gprefix = (int)o;
    o = align_up(o + sizeof(int) * T, 256);
    bytes = o;
}

static int klt_grid(const vt_batch *b, int win, int gtype) {
    const KltBatchKernel kb = klt_batch_kernel(win, gtype, b->klt_warps);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)kb.fn, b->klt_warps * 32, kb.smem);
    if (occ < 1) occ = 1;
    const int per = b->klt_ctas_per_sm > 0 && b->klt_ctas_per_sm < occ ? b->klt_ctas_per_sm : occ;
    return b->sms * per;
}

// ev (nullable): 4 events around the pyramid and tracking launches; lev
// (nullable): one event after each pyramid launch.
static vt_status enqueue(vt_batch *b, int k, cudaStream_t s, cudaEvent_t *ev = nullptr, cudaEvent_t *lev = nullptr) {
    const Topo &tp = b->topo[k];
    if (cudaMemcpyAsync(b->dev[k], b->host[k], b->tab_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(b->counter + k, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    if (ev && ev[0]) cudaEventRecord(ev[0], s);
    vt_status st = launch_pyr_batch(b->dev[k], tp.maxL, tp.gtype, tp.pyr_grid, b->tail_grid, s, lev);
    if (st != VT_OK) return st;
    if (ev && ev[1]) cudaEventRecord(ev[1], s);
    const KltBatchKernel kb = klt_batch_kernel(tp.win, tp.gtype, tp.klt_warps);
    if (!kb.fn) return VT_ERR_ARG;
    if (ev && ev[2]) cudaEventRecord(ev[2], s);
    // starts while the last pyramid launch finishes (programmatic dependent
    // launch), unless events are recorded for per-launch timing
    const cudaError_t e =
        launch_pdl(kb.fn, tp.klt_grid, tp.klt_warps * 32, kb.smem, s, !ev, (const uint8_t *)b->dev[k], b->counter + k);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return VT_ERR_CUDA;
    if (tp.fp64 && launch_klt_f64(b->dev[k], tp.win, tp.gtype, b->sms * 4, s) != VT_OK) return VT_ERR_CUDA;
    if (ev && ev[3]) cudaEventRecord(ev[3], s);
    if (tp.gate) return launch_gate_batch(b->dev[k], b->gate_grid, s);
    return VT_OK;
}

}  // namespace vt

extern "C" {

vt_status vt_batch_create(int max_frames, int max_tasks, vt_batch **out) {
    if (!out || max_frames < 0 || max_tasks < 0 || max_frames > (1 << 16) || max_tasks > (1 << 20)) return VT_ERR_ARG;
    vt_batch *b = (vt_batch *)calloc(1, sizeof(vt_batch));
    if (!b) return VT_ERR_OOM;
    b->cap_frames = max_frames > 0 ? max_frames : 1;
    b->cap_tasks = max_tasks > 0 ? max_tasks : 1;
    int of, oj, ots, ot, op, og, ogp;
    layout(b->cap_frames, b->cap_tasks, of, oj, ots, ot, op, og, ogp, b->tab_bytes);
    bool ok = true;
    for (int k = 0; k < 2; ++k) {
        ok = ok && cudaMallocHost((void **)&b->host[k], b->tab_bytes) == cudaSuccess;
        ok = ok && cudaMalloc((void **)&b->dev[k], b->tab_bytes) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&b->ev[k], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaMalloc((void **)&b->counter, 2 * sizeof(int)) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    ok = ok && cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        vt_batch_free(b);
        return VT_ERR_OOM;
    }
    b->klt_warps = 4;
    b->klt_ctas_per_sm = 0;
    b->tail_grid = 8 * b->cap_frames < 2 * b->sms ? 8 * b->cap_frames : 2 * b->sms;
    b->pyr_grid = b->sms * (pyr_batch_blocks_per_sm() > 0 ? pyr_batch_blocks_per_sm() : 1);
    b->gate_grid = 4 * b->sms;
    b->staged = -1;
    *out = b;
    return VT_OK;
}

void vt_batch_free(vt_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    for (int k = 0; k < 2; ++k) {
        for (int j = 0; j < kGraphsPerBuffer; ++j)
            if (b->exec[k][j]) cudaGraphExecDestroy(b->exec[k][j]);
        if (b->host[k]) cudaFreeHost(b->host[k]);
        if (b->dev[k]) cudaFree(b->dev[k]);
        if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    }
    if (b->counter) cudaFree(b->counter);
    if (b->cap) cudaStreamDestroy(b->cap);
    free(b);
}

vt_status vt_batch_config(vt_batch *b, int klt_warps_per_cta, int klt_ctas_per_sm, int pyr_ctas) {
    if (!b || (klt_warps_per_cta != 4 && klt_warps_per_cta != 8) || klt_ctas_per_sm < 0 || pyr_ctas < 0)
        return VT_ERR_ARG;
    b->klt_warps = klt_warps_per_cta;
    b->klt_ctas_per_sm = klt_ctas_per_sm;
    const int occ = pyr_batch_blocks_per_sm() > 0 ? pyr_batch_blocks_per_sm() : 1;
    b->pyr_grid = pyr_ctas > 0 ? pyr_ctas : b->sms * occ;
    return VT_OK;
}

vt_status vt_batch_set(vt_batch *b, const vt_frame_job *frames, int nframes, vt_grad_type gtype,
                       const vt_track_task *tasks, int ntasks, const vt_klt_params *prm) {
    if (!b || !prm || nframes < 0 || ntasks < 0 || nframes > b->cap_frames || ntasks > b->cap_tasks)
        return VT_ERR_ARG;
    if ((nframes > 0 && !frames) || (ntasks > 0 && !tasks)) return VT_ERR_ARG;
    if (gtype != VT_GRAD_S16 && gtype != VT_GRAD_F16 && gtype != VT_GRAD_NONE) return VT_ERR_ARG;
    if (!window_supported(prm->win) || prm->levels < 0 || prm->levels > VT_MAX_LEVELS || prm->max_iters < 1 ||
        !(prm->eps >= 0.f) || !(prm->min_eig >= 0.f) || !(prm->fb_thr >= 0.f))
        return VT_ERR_ARG;
    // validate everything before touching the staging buffer
    for (int f = 0; f < nframes; ++f) {
        const vt_frame_job &fj = frames[f];
        if (!fj.img || !fj.pyr || fj.pitch < fj.pyr->w) return VT_ERR_ARG;
        if (fj.img == fj.pyr->lv[0].img && fj.pitch != fj.pyr->lv[0].pitch) return VT_ERR_ARG;  // in place
        for (int g = 0; g < f; ++g)
            if (frames[g].pyr == fj.pyr) return VT_ERR_ARG;  // one build per pyramid per run
    }
    for (int t = 0; t < ntasks; ++t) {
        const vt_track_task &tk = tasks[t];
        if (!tk.prev || !tk.cur || tk.n < 0 || (tk.n > 0 && (!tk.pts_in || !tk.pts_out || !tk.status)))
            return VT_ERR_ARG;
        const int L = tk.levels > 0 ? tk.levels : prm->levels;
        if (tk.levels < 0 || L > tk.prev->levels || L > tk.cur->levels) return VT_ERR_ARG;
        auto gt_after = [&](const vt_pyramid *p) {
            for (int f = 0; f < nframes; ++f)
                if (frames[f].pyr == p) return (int)gtype;
            return p->gtype;
        };
        if (gt_after(tk.prev) != (int)gtype || (tk.fb && gt_after(tk.cur) != (int)gtype)) return VT_ERR_ARG;
    }
    const int k = b->next;
    if (b->ev_used[k]) {
        if (cudaEventSynchronize(b->ev[k]) != cudaSuccess) {
            cudaGetLastError();
            return VT_ERR_CUDA;
        }
    }
    uint8_t *tab = b->host[k];
    BatchHdr *H = reinterpret_cast<BatchHdr *>(tab);
    memset(H, 0, sizeof(BatchHdr));
    size_t bytes;
    layout(b->cap_frames, b->cap_tasks, H->off_frames, H->off_jobs, H->off_tsrc, H->off_tasks, H->off_prefix,
           H->off_gates, H->off_gprefix, bytes);
    H->cap_frames = b->cap_frames;
    H->cap_tasks = b->cap_tasks;
    H->nframes = nframes;
    H->ntasks = ntasks;
    H->P.win = prm->win;
    H->P.levels = prm->levels;
    H->P.max_iters = prm->max_iters;
    H->P.eps2 = prm->eps * prm->eps;
    H->P.min_eig = prm->min_eig;
    H->P.fb_thr2 = prm->fb_thr * prm->fb_thr;
    H->P.fp64 = fp64_needed(prm->min_eig);
    BFrame *bf = reinterpret_cast<BFrame *>(tab + H->off_frames);
    BLvlJob *jobs = reinterpret_cast<BLvlJob *>(tab + H->off_jobs);
    BTileSrc *tsrc = reinterpret_cast<BTileSrc *>(tab + H->off_tsrc);
    int maxL = 1, maxC = 0;
    for (int f = 0; f < nframes; ++f) {
        const vt_frame_job &fj = frames[f];
        vt_pyramid *p = fj.pyr;
        bf[f].img = fj.img;
        bf[f].lv = p->dev_lv;
        bf[f].pitch = fj.pitch;
        bf[f].vec_ok = ((uintptr_t)fj.img % 16 == 0) && (fj.pitch % 16 == 0);
        bf[f].levels = p->levels;
        p->gtype = (int)gtype;
        if (p->levels > maxL) maxL = p->levels;
        const int c = tail_start_level(p);
        if (c > maxC) maxC = c;
    }
    for (int l = 0; l < VT_MAX_LEVELS; ++l) {
        BLvlJob *lj = jobs + (size_t)l * b->cap_frames;
        int nj = 0, tiles = 0;
        for (int f = 0; f < nframes; ++f) {
            const vt_pyramid *p = frames[f].pyr;
            const int c = tail_start_level(p);
            if (l < VT_MAX_LEVELS - 1) {
                if (l >= c) continue;  // levels from c on are built by the tail kernel
                int tx = 0;
                const int nt = pyr_tiles(p->lv[l].w, p->lv[l].h, tx);
                lj[nj].frame = f;
                lj[nj].tiles_x = tx;
                lj[nj].tile0 = tiles;
                lj[nj].aux = c;
                BTileSrc &ts = tsrc[(size_t)l * b->cap_frames + nj];
                const Level &S = p->lv[l], &D = p->lv[l + 1];
                ts.src = l == 0 ? frames[f].img : S.img;
                ts.spitch = l == 0 ? frames[f].pitch : S.pitch;
                ts.vec_ok = l == 0 ? bf[f].vec_ok : 1;
                ts.w = S.w;
                ts.h = S.h;
                ts.dst = D.img;
                ts.dpitch = D.pitch;
                ts.grad = S.grad;
                ts.gpitch = S.gpitch;
                // level 0 also writes the pyramid's own level-0 copy, unless
                // the frame is built in place (its image is that level)
                ts.copy = (l == 0 && frames[f].img != S.img) ? S.img : nullptr;
                ts.cpitch = S.pitch;
                ts.tiles_x = tx;
                tiles += nt;
                ++nj;
            } else {
                // bands per frame capped so that every band of the run gets a
                // CTA of the tail launch in one round
                const int cap = b->tail_grid / (nframes > 0 ? nframes : 1);
                int parts = tail_parts(p);
                if (parts > cap) parts = cap > 1 ? cap : 1;
                for (int q = 0; q < parts; ++q) {
                    lj[nj].frame = f;
                    lj[nj].tiles_x = q;
                    lj[nj].tile0 = parts;
                    lj[nj].aux = c;
                    ++nj;
                    ++tiles;
                }
            }
        }
        H->njobs[l] = nj;
        H->ntiles[l] = tiles;
    }
    BTask *bt = reinterpret_cast<BTask *>(tab + H->off_tasks);
    int *p0s = reinterpret_cast<int *>(tab + H->off_prefix);
    long total = 0;
    for (int t = 0; t < ntasks; ++t) {
        const vt_track_task &tk = tasks[t];
        bt[t].I = tk.prev->dev_lv;
        bt[t].J = tk.cur->dev_lv;
        bt[t].pts_in = reinterpret_cast<const float2 *>(tk.pts_in);
        bt[t].pts_out = reinterpret_cast<float2 *>(tk.pts_out);
        bt[t].status = tk.status;
        bt[t].err = tk.err;
        bt[t].reason = tk.reason;
        bt[t].flops = tk.flops;
        bt[t].n_dev = tk.n_dev;
        bt[t].n = tk.n;
        bt[t].fb = tk.fb ? 1 : 0;
        bt[t].levels = tk.levels > 0 ? tk.levels : prm->levels;
        bt[t].p0 = (int)total;
        p0s[t] = (int)total;
        total += tk.n;
    }
    if (total > 0x7fffffff) return VT_ERR_ARG;
    H->total_points = (int)total;
    H->maxL = maxL;
    Topo &tp = b->topo[k];
    tp.maxL = maxC;  // tiled pyramid launches of this run
    tp.gtype = (int)gtype;
    tp.win = prm->win;
    tp.klt_warps = b->klt_warps;
    tp.klt_grid = klt_grid(b, prm->win, (int)gtype);
    tp.pyr_grid = b->pyr_grid;
    tp.gate = 0;
    tp.fp64 = H->P.fp64;
    b->staged = k;
    b->next = k ^ 1;
    b->fresh = true;
    return VT_OK;
}

vt_status vt_batch_set_gates(vt_batch *b, const vt_gate_task *gates, int ngates, const vt_gate_params *prm) {
    if (!b || b->staged < 0 || !b->fresh || ngates < 0 || ngates > b->cap_tasks || (ngates > 0 && !gates))
        return VT_ERR_ARG;
    for (int i = 0; i < ngates; ++i) {
        const vt_gate_task &g = gates[i];
        if (g.n < 0 || !gate_args_ok(&g.rig, prm) || (g.n > 0 && (!g.pts_l || !g.pts_r || !g.status_out)))
            return VT_ERR_ARG;
    }
    const int k = b->staged;
    uint8_t *tab = b->host[k];
    BatchHdr *H = reinterpret_cast<BatchHdr *>(tab);
    GTask *gt = reinterpret_cast<GTask *>(tab + H->off_gates);
    int *p0s = reinterpret_cast<int *>(tab + H->off_gprefix);
    long total = 0;
    for (int i = 0; i < ngates; ++i) {
        const vt_gate_task &g = gates[i];
        gt[i].rig = g.rig;
        gt[i].pts_l = reinterpret_cast<const float2 *>(g.pts_l);
        gt[i].pts_r = reinterpret_cast<const float2 *>(g.pts_r);
        gt[i].status_in = g.status_in;
        gt[i].xyz = g.xyz;
        gt[i].status_out = g.status_out;
        gt[i].reason = g.reason;
        gt[i].n = g.n;
        gt[i].p0 = (int)total;
        p0s[i] = (int)total;
        total += g.n;
    }
    if (total > 0x7fffffff) return VT_ERR_ARG;
    H->ngates = ngates;
    H->gate_points = (int)total;
    if (prm) H->G = *prm;
    b->topo[k].gate = ngates > 0 ? 1 : 0;
    return VT_OK;
}

vt_status vt_batch_run(vt_batch *b, void *cuda_stream) {
    if (!b || b->staged < 0) return VT_ERR_ARG;
    const int k = b->staged;
    b->fresh = false;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    vt_status st = enqueue(b, k, s);
    if (st != VT_OK) return st;
    if (cudaEventRecord(b->ev[k], s) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    b->ev_used[k] = true;
    return VT_OK;
}

vt_status vt_batch_run_timed(vt_batch *b, void *cuda_stream, void *ev_pyr0, void *ev_pyr1, void *ev_klt0,
                             void *ev_klt1) {
    if (!b || b->staged < 0) return VT_ERR_ARG;
    const int k = b->staged;
    b->fresh = false;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t ev[4] = {(cudaEvent_t)ev_pyr0, (cudaEvent_t)ev_pyr1, (cudaEvent_t)ev_klt0, (cudaEvent_t)ev_klt1};
    vt_status st = enqueue(b, k, s, ev);
    if (st != VT_OK) return st;
    if (cudaEventRecord(b->ev[k], s) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    b->ev_used[k] = true;
    return VT_OK;
}

vt_status vt_batch_run_levels_timed(vt_batch *b, void *cuda_stream, void **events, int nevents) {
    if (!b || b->staged < 0 || !events || nevents < 0) return VT_ERR_ARG;
    const int k = b->staged;
    const int need = b->topo[k].maxL + 1 + 4;
    if (nevents < need) return VT_ERR_ARG;
    b->fresh = false;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t ev[4] = {(cudaEvent_t)events[0], (cudaEvent_t)events[1], (cudaEvent_t)events[2],
                         (cudaEvent_t)events[3]};
    vt_status st = enqueue(b, k, s, ev, reinterpret_cast<cudaEvent_t *>(events + 4));
    if (st != VT_OK) return st;
    if (cudaEventRecord(b->ev[k], s) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    b->ev_used[k] = true;
    return VT_OK;
}

vt_status vt_batch_run_graph(vt_batch *b, void *cuda_stream) {
    if (!b || b->staged < 0) return VT_ERR_ARG;
    const int k = b->staged;
    b->fresh = false;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int slot = -1;
    for (int j = 0; j < kGraphsPerBuffer && slot < 0; ++j)
        if (b->exec[k][j] && b->exec_topo[k][j] == b->topo[k]) slot = j;
    if (slot < 0) {
        slot = b->exec_next[k];
        b->exec_next[k] = (slot + 1) % kGraphsPerBuffer;
        if (b->exec[k][slot]) {
            cudaGraphExecDestroy(b->exec[k][slot]);
            b->exec[k][slot] = nullptr;
        }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return VT_ERR_CUDA;
        }
        vt_status st = enqueue(b, k, b->cap);
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (st != VT_OK || e != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            return st != VT_OK ? st : VT_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&b->exec[k][slot], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->exec[k][slot] = nullptr;
            return VT_ERR_CUDA;
        }
        b->exec_topo[k][slot] = b->topo[k];
    }
    if (cudaGraphLaunch(b->exec[k][slot], s) != cudaSuccess || cudaEventRecord(b->ev[k], s) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    b->ev_used[k] = true;
    return VT_OK;
}

vt_status vt_copy_async(const vt_copy *copies, int n, void *cuda_stream) {
    if (n < 0 || (n > 0 && !copies)) return VT_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (copies[i].bytes && (!copies[i].dst || !copies[i].src)) return VT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    for (int i = 0; i < n; ++i) {
        if (!copies[i].bytes) continue;
        if (cudaMemcpyAsync(copies[i].dst, copies[i].src, copies[i].bytes, cudaMemcpyDefault, s) != cudaSuccess) {
            cudaGetLastError();
            return VT_ERR_CUDA;
        }
    }
    return VT_OK;
}

vt_status vt_batch_info(const vt_batch *b, int *klt_grid_ctas, int *klt_warps_per_cta, int *pyr_grid_ctas,
                        int *launches_per_run) {
    if (!b) return VT_ERR_ARG;
    const int k = b->staged >= 0 ? b->staged : 0;
    if (klt_grid_ctas) *klt_grid_ctas = b->topo[k].klt_grid;
    if (klt_warps_per_cta) *klt_warps_per_cta = b->topo[k].klt_warps;
    if (pyr_grid_ctas) *pyr_grid_ctas = b->topo[k].pyr_grid;
    if (launches_per_run)
        *launches_per_run = b->staged >= 0 ? b->topo[k].maxL + 1 + 1 + b->topo[k].fp64 + b->topo[k].gate : 0;
    return VT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Tracking of many tasks without any allocation.
//
// Some callers cannot allocate device memory at call time: real-time loops
// that must not block on the allocator or on the device-wide synchronisation
// cudaFree can cause, and hosts (frameworks, plug-in hosts) that hand out all
// device memory from their own pools.  For them the tracking launch of
// vt_batch can run with its job table and work counter in the file-scope
// array below instead of a vt_batch's allocations.  The table travels to the
// device as a kernel parameter (a snapshot taken at the launch), so no host
// buffer has to outlive the call.
namespace vt {

constexpr int kNoAllocMaxTasks = 256;
constexpr size_t kNoAllocTaskOff = 256;  // after a BatchHdr (checked below)
constexpr size_t kNoAllocPrefixOff = kNoAllocTaskOff + sizeof(BTask) * kNoAllocMaxTasks;
constexpr size_t kNoAllocCounterOff = (kNoAllocPrefixOff + sizeof(int) * kNoAllocMaxTasks + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kNoAllocCounterOff + 256;
static_assert(sizeof(BatchHdr) <= kNoAllocTaskOff, "header must fit before the task table");
static_assert(kNoAllocBytes == 24064, "the size vt.h states");

// Shared by every call on a device; kept until the process exits.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

// The job table of one call, passed by value to k_noalloc_fill.
struct NoAllocTable {
    BatchHdr hdr;
    BTask tasks[kNoAllocMaxTasks];
    int prefix[kNoAllocMaxTasks];
};
static_assert(sizeof(NoAllocTable) <= 32000, "the table must fit the kernel-parameter limit");

// Writes the header, the first `ntasks` tasks and prefix entries into the
// scratch array and zeroes the work counter.  One CTA.
__global__ void k_noalloc_fill(const __grid_constant__ NoAllocTable T) {
    uint8_t *base = g_noalloc_scratch;
    const int nt = T.hdr.ntasks;
    const uint32_t *hs = reinterpret_cast<const uint32_t *>(&T.hdr);
    uint32_t *hd = reinterpret_cast<uint32_t *>(base);
    for (int i = threadIdx.x; i < (int)(sizeof(BatchHdr) / 4); i += blockDim.x) hd[i] = hs[i];
    const uint32_t *ts = reinterpret_cast<const uint32_t *>(T.tasks);
    uint32_t *td = reinterpret_cast<uint32_t *>(base + kNoAllocTaskOff);
    const int tw = nt * (int)(sizeof(BTask) / 4);
    for (int i = threadIdx.x; i < tw; i += blockDim.x) td[i] = ts[i];
    int *pd = reinterpret_cast<int *>(base + kNoAllocPrefixOff);
    for (int i = threadIdx.x; i < nt; i += blockDim.x) pd[i] = T.prefix[i];
    if (threadIdx.x == 0) *reinterpret_cast<int *>(base + kNoAllocCounterOff) = 0;
}
static_assert(sizeof(BatchHdr) % 4 == 0 && sizeof(BTask) % 4 == 0, "word copies");

constexpr int kNoAllocMaxDevices = 64;
static std::atomic<uint8_t *> g_noalloc_ptr[kNoAllocMaxDevices];

// Device address of the scratch array on the current device, looked up on
// the first call per device (the array's host-side name is not an address).
// Threads racing on a first call look it up twice and store the same value.
static vt_status noalloc_scratch(uint8_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    uint8_t *p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void *q = nullptr;
        if (cudaGetSymbolAddress(&q, g_noalloc_scratch) != cudaSuccess || !q) {
            cudaGetLastError();
            return VT_ERR_CUDA;
        }
        p = (uint8_t *)q;
        g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return VT_OK;
}

}  // namespace vt

extern "C" vt_status vt_klt_track_tasks_noalloc(const vt_track_task *tasks, int ntasks, const vt_klt_params *prm,
                                                void *cuda_stream) {
    if (!prm || ntasks < 0 || (ntasks > 0 && !tasks)) return VT_ERR_ARG;
    if (ntasks > kNoAllocMaxTasks) return VT_ERR_ARG;  // beyond the fixed table
    if (!window_supported(prm->win) || prm->levels < 0 || prm->levels > VT_MAX_LEVELS || prm->max_iters < 1 ||
        !(prm->eps >= 0.f) || !(prm->min_eig >= 0.f) || !(prm->fb_thr >= 0.f))
        return VT_ERR_ARG;
    if (ntasks == 0) return VT_OK;
    if (!tasks[0].prev) return VT_ERR_ARG;
    const int gtype = tasks[0].prev->gtype;  // VT_GRAD_NONE: gradients computed in the tracker
    long total = 0;
    for (int t = 0; t < ntasks; ++t) {
        const vt_track_task &tk = tasks[t];
        if (!tk.prev || !tk.cur || tk.n < 0 || (tk.n > 0 && (!tk.pts_in || !tk.pts_out || !tk.status)))
            return VT_ERR_ARG;
        const int L = tk.levels > 0 ? tk.levels : prm->levels;
        if (tk.levels < 0 || L < 1 || L > tk.prev->levels || L > tk.cur->levels) return VT_ERR_ARG;
        if (tk.prev->gtype != gtype || (tk.fb && tk.cur->gtype != gtype)) return VT_ERR_ARG;
        total += tk.n;
    }
    if (total > 0x7fffffff) return VT_ERR_ARG;
    if (total == 0) return VT_OK;
    const KltBatchKernel kb = klt_batch_kernel(prm->win, gtype, 4);
    if (!kb.fn) return VT_ERR_ARG;
    uint8_t *dev = nullptr;
    vt_status st = noalloc_scratch(&dev);
    if (st != VT_OK) return st;
    // the job table, built here and handed to the fill kernel by value
    static thread_local NoAllocTable T;
    memset(&T.hdr, 0, sizeof(T.hdr));
    BatchHdr *H = &T.hdr;
    H->ntasks = ntasks;
    H->total_points = (int)total;
    H->off_tasks = (int)kNoAllocTaskOff;
    H->off_prefix = (int)kNoAllocPrefixOff;
    H->P.win = prm->win;
    H->P.levels = prm->levels;
    H->P.max_iters = prm->max_iters;
    H->P.eps2 = prm->eps * prm->eps;
    H->P.min_eig = prm->min_eig;
    H->P.fb_thr2 = prm->fb_thr * prm->fb_thr;
    H->P.fp64 = fp64_needed(prm->min_eig);
    int p0 = 0;
    for (int t = 0; t < ntasks; ++t) {
        const vt_track_task &tk = tasks[t];
        BTask &b = T.tasks[t];
        b.I = tk.prev->dev_lv;
        b.J = tk.cur->dev_lv;
        b.pts_in = reinterpret_cast<const float2 *>(tk.pts_in);
        b.pts_out = reinterpret_cast<float2 *>(tk.pts_out);
        b.status = tk.status;
        b.err = tk.err;
        b.reason = tk.reason;
        b.flops = tk.flops;
        b.n_dev = tk.n_dev;
        b.n = tk.n;
        b.fb = tk.fb ? 1 : 0;
        b.levels = tk.levels > 0 ? tk.levels : prm->levels;
        b.p0 = p0;
        T.prefix[t] = p0;
        p0 += tk.n;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_noalloc_fill<<<1, 256, 0, s>>>(T);
    int sms = 0, occ = 0, d = 0;
    cudaGetDevice(&d);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)kb.fn, 4 * 32, kb.smem);
    if (sms < 1) sms = 1;
    if (occ < 1) occ = 1;
    kb.fn<<<sms * occ, 4 * 32, kb.smem, s>>>(dev, reinterpret_cast<int *>(dev + kNoAllocCounterOff));
    if (cudaGetLastError() != cudaSuccess) return VT_ERR_CUDA;
    return T.hdr.P.fp64 ? launch_klt_f64(dev, prm->win, gtype, sms * 4, s) : VT_OK;
}
