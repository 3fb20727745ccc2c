// Single-pair tracking kernels and their C ABI: vt_klt_track, vt_klt_track_ex,
// vt_klt_track_fb (forward + backward + FB test fused per warp) and
// vt_fb_check (K4).  The per-point arithmetic is in vt_klt.cuh.
#include "vt_klt.cuh"

namespace vt {

constexpr int KLT_WARPS = 4;  // warps (points) per CTA

struct KltArgs {
    KPyr I, J;
    const float2 *pts_in;
    const float2 *guess;
    int n;
    float2 *pts_out;
    uint8_t *status;
    float *err;
    uint8_t *reason;
    int32_t *iters;
    float *lmin;
    int32_t *flops;
    int32_t *sweeps;
    KParams P;
};

// F64 = false: the FP32 tracker; a point with an ill-conditioned level is
// left pending (status kStatusPending).  F64 = true: the second launch,
// which tracks only the pending points, with such levels in FP64.
template <int WIN, int GT, bool FB, bool F64>
__global__ void __launch_bounds__(KLT_WARPS * 32, KltOcc<WIN>::min_blocks) k_klt(const __grid_constant__ KltArgs A) {
    extern __shared__ __align__(16) uint8_t klt_smem[];
    KSmem<WIN> &sm = reinterpret_cast<KSmem<WIN> *>(klt_smem)[threadIdx.x >> 5];
    ksmem_init<WIN>(sm, threadIdx.x & 31);
    const int pt = blockIdx.x * KLT_WARPS + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (pt >= A.n) return;
    if (F64 && A.status[pt] != kStatusPending) return;
    const float2 p = A.pts_in[pt];
    KOut o;
    float2 g = make_float2(0.f, 0.f);
    const bool hg = !FB && A.guess != nullptr;
    if (hg) g = A.guess[pt];
    track_point_dir<WIN, GT, F64>(A.I.lv, A.J.lv, A.P, p.x, p.y, FB, hg, g.x, g.y, lane, sm, o);
    if (!F64 && o.reason == kReasonPending) {
        if (lane == 0) A.status[pt] = kStatusPending;
        return;
    }
    if (lane == 0) {
        A.pts_out[pt] = make_float2(o.x, o.y);
        A.status[pt] = (uint8_t)o.status;
        if (A.err) A.err[pt] = o.status ? o.err : 0.f;
        if (A.reason) A.reason[pt] = (uint8_t)o.reason;
        if (A.iters) A.iters[pt] = o.iters;
        if (A.lmin) A.lmin[pt] = o.lmin;
        if (A.flops) A.flops[pt] = klt_flops(WIN, o);
        if (A.sweeps) A.sweeps[pt] = o.sweeps;
    }
}

__global__ void k_fb_check(const float2 *p0, const float2 *p1, const uint8_t *sf, const uint8_t *sb, int n,
                           float thr2, uint8_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 a = p0[i], b = p1[i];
    const float dx = a.x - b.x, dy = a.y - b.y;
    out[i] = (uint8_t)(sf[i] && sb[i] && (dx * dx + dy * dy <= thr2));
}

template <int WIN, int GT, bool FB, bool F64>
static void launch_pass(const KltArgs &A, cudaStream_t s) {
    const int blocks = (A.n + KLT_WARPS - 1) / KLT_WARPS;
    const size_t smem = KLT_WARPS * sizeof(KSmem<WIN>);
    if (smem > 48 * 1024) {
        static const bool attr = [smem] {  // once, thread-safe static initialisation
            return cudaFuncSetAttribute(k_klt<WIN, GT, FB, F64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem) == cudaSuccess;
        }();
        (void)attr;
    }
    k_klt<WIN, GT, FB, F64><<<blocks, KLT_WARPS * 32, smem, s>>>(A);
}

// The FP32 launch, then (only when an accepted template can be
// ill-conditioned, fp64_needed) the FP64-capable launch over its pending points.
template <int WIN, int GT, bool FB>
static vt_status launch_one(const KltArgs &A, cudaStream_t s) {
    launch_pass<WIN, GT, FB, false>(A, s);
    if (A.P.fp64) launch_pass<WIN, GT, FB, true>(A, s);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

template <int GT, bool FB>
static vt_status dispatch_win(const KltArgs &A, cudaStream_t s) {
    switch (A.P.win) {
        case 9: return launch_one<9, GT, FB>(A, s);
        case 15: return launch_one<15, GT, FB>(A, s);
        case 21: return launch_one<21, GT, FB>(A, s);
        case 31: return launch_one<31, GT, FB>(A, s);
    }
    return VT_ERR_ARG;
}

bool window_supported(int win) { return win == 9 || win == 15 || win == 21 || win == 31; }

static void fill_pyr(KPyr &K, const vt_pyramid *p) {
    for (int l = 0; l < VT_MAX_LEVELS; ++l) K.lv[l] = l < p->levels ? p->lv[l] : Level{};
}

static vt_status track_common(const vt_pyramid *prev, const vt_pyramid *cur, const float *pts_in, int n,
                              const float *pts_guess, const vt_klt_params *prm, float *pts_out, uint8_t *status,
                              float *err, const vt_klt_diag *diag, bool fb, void *cuda_stream) {
    if (!prev || !cur || !prm || n < 0) return VT_ERR_ARG;
    if (n > 0 && (!pts_in || !pts_out || !status)) return VT_ERR_ARG;
    if (!window_supported(prm->win)) return VT_ERR_ARG;
    if (prm->levels < 1 || prm->levels > prev->levels || prm->levels > cur->levels) return VT_ERR_ARG;
    if (prm->max_iters < 1 || !(prm->eps >= 0.f) || !(prm->min_eig >= 0.f)) return VT_ERR_ARG;
    if (fb && !(prm->fb_thr >= 0.f)) return VT_ERR_ARG;
    if (fb && cur->gtype != prev->gtype) return VT_ERR_ARG;
    if (n == 0) return VT_OK;
    KltArgs A;
    fill_pyr(A.I, prev);
    fill_pyr(A.J, cur);
    A.pts_in = reinterpret_cast<const float2 *>(pts_in);
    A.guess = reinterpret_cast<const float2 *>(pts_guess);
    A.n = n;
    A.pts_out = reinterpret_cast<float2 *>(pts_out);
    A.status = status;
    A.err = err;
    A.reason = diag ? diag->reason : nullptr;
    A.iters = diag ? diag->iters : nullptr;
    A.lmin = diag ? diag->lmin : nullptr;
    A.flops = diag ? diag->flops : nullptr;
    A.sweeps = diag ? diag->sweeps : nullptr;
    A.P.win = prm->win;
    A.P.levels = prm->levels;
    A.P.max_iters = prm->max_iters;
    A.P.eps2 = prm->eps * prm->eps;
    A.P.min_eig = prm->min_eig;
    A.P.fb_thr2 = prm->fb_thr * prm->fb_thr;
    A.P.fp64 = fp64_needed(prm->min_eig);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (prev->gtype == VT_GRAD_F16)
        return fb ? dispatch_win<VT_GRAD_F16, true>(A, s) : dispatch_win<VT_GRAD_F16, false>(A, s);
    if (prev->gtype == VT_GRAD_NONE)  // gradients computed in the tracker, as int16 Scharr
        return fb ? dispatch_win<VT_GRAD_NONE, true>(A, s) : dispatch_win<VT_GRAD_NONE, false>(A, s);
    return fb ? dispatch_win<VT_GRAD_S16, true>(A, s) : dispatch_win<VT_GRAD_S16, false>(A, s);
}

}  // namespace vt

using namespace vt;

extern "C" {

vt_status vt_klt_track(const vt_pyramid *prev, const vt_pyramid *cur, const float *pts_in, int n,
                       const float *pts_guess, int win, int levels, int max_iters, float eps, float *pts_out,
                       uint8_t *status, float *err, void *cuda_stream) {
    vt_klt_params p{win, levels, max_iters, eps, VT_DEFAULT_MIN_EIG, 0.f};
    return track_common(prev, cur, pts_in, n, pts_guess, &p, pts_out, status, err, nullptr, false, cuda_stream);
}

vt_status vt_klt_track_ex(const vt_pyramid *prev, const vt_pyramid *cur, const float *pts_in, int n,
                          const float *pts_guess, const vt_klt_params *prm, float *pts_out, uint8_t *status,
                          float *err, const vt_klt_diag *diag, void *cuda_stream) {
    return track_common(prev, cur, pts_in, n, pts_guess, prm, pts_out, status, err, diag, false, cuda_stream);
}

vt_status vt_klt_track_fb(const vt_pyramid *prev, const vt_pyramid *cur, const float *pts_in, int n,
                          const vt_klt_params *prm, float *pts_out, uint8_t *status, float *err,
                          const vt_klt_diag *diag, void *cuda_stream) {
    return track_common(prev, cur, pts_in, n, nullptr, prm, pts_out, status, err, diag, true, cuda_stream);
}

vt_status vt_fb_check(const float *p0, const float *p0_back, const uint8_t *st_f, const uint8_t *st_b, int n,
                      float thr, uint8_t *status_out, void *cuda_stream) {
    if (n < 0 || !(thr >= 0.f)) return VT_ERR_ARG;
    if (n == 0) return VT_OK;
    if (!p0 || !p0_back || !st_f || !st_b || !status_out) return VT_ERR_ARG;
    const int threads = 256;
    k_fb_check<<<(n + threads - 1) / threads, threads, 0, (cudaStream_t)cuda_stream>>>(
        reinterpret_cast<const float2 *>(p0), reinterpret_cast<const float2 *>(p0_back), st_f, st_b, n, thr * thr,
        status_out);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// FP32 FMA throughput probe: the denominator of the tracking kernel's
// roofline is this device's measured FMA rate rather than a data-sheet figure.
// Every thread runs 8 independent FMA chains (enough independent work per
// warp to keep the FMA pipes issuing at full occupancy), 8 x iters FMAs of
// 2 FLOPs each, and writes one sum so nothing is optimised away.
namespace vt {

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 8;  // 2048 threads per SM

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float *out, int iters, float m, float c) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace vt

extern "C" vt_status vt_fp32_fma_probe(int iters, float *out, long long out_floats, long long *flops,
                                       void *cuda_stream) {
    int dev = 0, sms = 0;
    if (iters < 1 || !out || !flops || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_ARG;
    }
    const long long grid = (long long)sms * kProbeCtasPerSm;
    if (out_floats < grid * kProbeThreads) return VT_ERR_ARG;
    vt::k_fma_probe<<<(int)grid, kProbeThreads, 0, (cudaStream_t)cuda_stream>>>(out, iters, 0.999f, 1e-3f);
    *flops = grid * kProbeThreads * 8LL * 8LL * iters * 2LL;
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}
