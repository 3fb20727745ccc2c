// Internal structures shared by the CUDA translation units of libvt.
// Device-side layout of a pyramid, job tables and small device helpers.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vt.h"

namespace vt {

// One level as the kernels see it.  Images are uint8 with `pitch` bytes per
// row (multiple of 64); gradients are 32-bit (dx, dy) pairs (int16x2 or
// half2) with `gpitch` pairs per row (multiple of 32, i.e. 128-byte rows).
struct Level {
    uint8_t *img;
    uint32_t *grad;
    int w, h, pitch, gpitch;
};

}  // namespace vt

struct vt_pyramid {
    int w, h, levels;
    int gtype;  // vt_grad_type of the current gradient planes
    int device;
    void *base;  // single device allocation holding every level and plane
    size_t bytes;
    vt::Level lv[VT_MAX_LEVELS];
    vt::Level *dev_lv;  // device copy of lv[] (written once at allocation)
};

namespace vt {

constexpr int kImgPitchAlign = 64;
constexpr int kGradPitchAlign = 32;

inline int round_up(int v, int a) { return (v + a - 1) / a * a; }

// Reflect-101 border index; a 1-px side clamps.
__device__ __forceinline__ int refl101(int i, int n) {
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * n - 2 - i;
    }
    return i;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation (launch_pdl) may start before the previous kernel on its
// stream has finished: it reads only what was ready before that kernel began
// (job tables) until pdl_wait() returns, which happens once the previous
// kernel has completed and its writes are visible.  pdl_trigger() lets the
// next such kernel start launching (its CTAs fill the SMs this kernel's
// finished CTAs leave).  Both are no-ops for a normally launched kernel.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Launch `k` on stream `s`, with programmatic stream serialisation when
// `pdl` (the kernel must call pdl_wait() before it reads the previous
// kernel's output).
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*k)(Params...), int grid, int block, size_t smem, cudaStream_t s, bool pdl,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// ---------------------------------------------------------------- pyramid jobs
// A pyrDown (and optionally Scharr) job: level src (w x h) -> dst
// (ceil(w/2) x ceil(h/2)); gradients of the src level when grad != nullptr.
struct PyrJob {
    const uint8_t *src;
    uint8_t *dst;
    uint32_t *grad;
    int w, h, spitch, dpitch, gpitch;
    int tiles_x;  // output tiles along x
    int tile0;    // first block of this job
};

constexpr int kMaxJobs = 48;

struct PyrJobs {
    int njobs;
    PyrJob j[kMaxJobs];
};

// A Scharr-only job over one level.
struct GradJob {
    const uint8_t *src;
    uint32_t *grad;
    int w, h, spitch, gpitch;
    int tiles_x;
    int tile0;
};

struct GradJobs {
    int njobs;
    GradJob j[kMaxJobs];
};

// Tracking parameters as the kernels use them.
struct KParams {
    int win, levels, max_iters;
    float eps2;     // eps^2
    float min_eig;  // threshold on lambda_min / (win^2 255^2)
    float fb_thr2;  // fb_thr^2
    int fp64;       // ill-conditioned levels go to the FP64-capable launch (see fp64_needed)
};

// Threshold on lambda_max / lambda_min of a level's gradient matrix above
// which the level is decided and tracked in FP64.
constexpr float kFp64Cond = 1e4f;

// Whether an accepted template can be ill-conditioned at all.  Bilinear
// samples of Scharr gradients are at most 4080/32 per component, so
// lambda_max <= win^2 * 2 * 127.5^2, while an accepted template has
// lambda_min >= min_eig * win^2 * 255^2: its condition number is at most
// 0.5 / min_eig.  Below kFp64Cond (min_eig >= 5e-5, the default 1e-4
// included) no level needs FP64 and the FP64-capable launch is skipped.
inline bool fp64_needed(float min_eig) { return !(min_eig * kFp64Cond >= 0.5f); }

// ------------------------------------------------------- batched job tables
// Device-side tables of one batched run (vt_batch): a header followed by the
// frame, per-level job, task and task-prefix arrays at the header's offsets.
struct BFrame {
    const uint8_t *img;  // caller image (level-0 source)
    const Level *lv;     // device level table of the destination pyramid
    int pitch;
    int vec_ok;  // img and pitch 16-byte aligned
    int levels;
    int pad;
};

// Everything a tile of one tiled pyramid job needs, resolved on the host
// when the tables are staged (no dependent loads of frame and level tables
// in the kernel): source level, destination level, gradient planes of the
// source level, and the level-0 copy destination (null when built in place).
struct __align__(16) BTileSrc {
    const uint8_t *src;
    uint8_t *dst;
    uint32_t *grad;
    uint8_t *copy;
    int w, h, spitch, dpitch, gpitch, cpitch, vec_ok, tiles_x;
};

struct BLvlJob {
    int frame;
    int tiles_x;
    int tile0;  // first tile of this job within its launch
    int aux;    // tail list: first level the tail kernel builds (c); in tail
                // lists tiles_x is the band index and tile0 the band count
};

// Levels of at most this many pixels are built by the tail kernel, one CTA
// per frame, entirely in shared memory.
constexpr int kTailMaxPx = 40960;

struct BTask {
    const Level *I;  // template pyramid (device level table)
    const Level *J;  // target pyramid
    const float2 *pts_in;
    float2 *pts_out;
    uint8_t *status;
    float *err;
    uint8_t *reason;
    int32_t *flops;
    const int *n_dev;  // nullable: device-side count (points beyond it are skipped)
    int n, fb, p0, levels;
};

// One stereo-gate task of a batched run: a rig and the pairs it checks.
struct GTask {
    vt_stereo_rig rig;
    const float2 *pts_l, *pts_r;
    const uint8_t *status_in;
    float *xyz;
    uint8_t *status_out, *reason;
    int n, p0;
};

struct BatchHdr {
    int nframes, ntasks, total_points, maxL;
    int njobs[VT_MAX_LEVELS];   // [l < VT_MAX_LEVELS-1]: tiled pyramid launch l; [VT_MAX_LEVELS-1]: tail jobs
    int ntiles[VT_MAX_LEVELS];
    int cap_frames, cap_tasks;
    int off_frames, off_jobs, off_tasks, off_prefix;
    int ngates, gate_points, off_gates, off_gprefix;
    int off_tsrc, pad_tsrc;  // BTileSrc per tiled job: VT_MAX_LEVELS - 1 lists of cap_frames
    vt_gate_params G;
    KParams P;
};

// Batched stereo gate (vt_stereo.cu): every gate task of the table at dev_tab,
// grid-stride over their pairs.
vt_status launch_gate_batch(const uint8_t *dev_tab, int grid, cudaStream_t s);
bool gate_args_ok(const vt_stereo_rig *rig, const vt_gate_params *prm);

// Host helpers implemented in vt_pyramid.cu.
// `ev` (nullable): one event recorded after each launch (tiled_launches + 1).
vt_status launch_pyr_batch(const uint8_t *dev_tab, int tiled_launches, int gtype, int grid_pyr, int grid_tail,
                           cudaStream_t s, cudaEvent_t *ev = nullptr);
int tail_start_level(const vt_pyramid *p);
int tail_parts(const vt_pyramid *p);
int pyr_batch_blocks_per_sm();
int pyr_tiles(int w, int h, int &tiles_x);
__host__ __device__ int scharr_tiles(int w, int h, int &tiles_x);
bool window_supported(int win);
vt_status launch_pyrdown(const PyrJobs &jobs, int total_blocks, int gtype, cudaStream_t s);
vt_status launch_scharr(const GradJobs &jobs, int total_blocks, int gtype, cudaStream_t s);
void add_pyr_job(PyrJobs &jobs, int &blocks, const Level &src, const Level &dst, bool with_grad);
void add_grad_job(GradJobs &jobs, int &blocks, const Level &lv);

}  // namespace vt
