// Stereo triangulation gate (K7): the per-point geometric check of stereo
// correspondences (Sec. III-C: negligible-disparity matches are dropped, the
// rest triangulated with the rig's extrinsics and kept only with a positive
// depth inside a valid range and at most 1.5 px of reprojection error in
// both views).  One thread per correspondence, FP64 throughout:
//
//   disparity  |p_R - pi_R(R K_L^-1 p_L)| (image of the left ray's point at
//              infinity in the right view; infinite when it lies behind the
//              right camera), kept when > min_disp;
//   DLT        the homogeneous point is the eigenvector of the smallest
//              eigenvalue of A^T A, A = [x_L P_L^3 - P_L^1; y_L P_L^3 - P_L^2;
//              x_R P_R^3 - P_R^1; y_R P_R^3 - P_R^2] on normalised
//              coordinates, P_L = [I | 0], P_R = [R | t]; cyclic Jacobi
//              rotations on the 4x4 (at most kJacobiSweeps sweeps);
//   depth      X_4 != 0, Z_R > 0, z_min <= Z_L <= z_max;
//   reprojection  both views' pixel errors <= max_reproj.
#include <cmath>
#include <cstdint>

#include "vt_internal.cuh"

namespace vt {

constexpr int kJacobiSweeps = 12;

struct GateArgs {
    vt_stereo_rig rig;
    vt_gate_params prm;
};

// One Jacobi rotation in the (P, Q) plane of the symmetric M (upper
// triangle M[i][j], i < j, and the diagonal are kept), accumulating V.
//
// GB300 issues FP64 at a small fraction of its FP32 rate, so the angle is
// found in FP32 (tan t, the smaller root of t^2 + 2 tau t - 1 = 0,
// tau = (M_QQ - M_PP) / 2 M_PQ) and only made exactly orthogonal in FP64:
// c = 1 / sqrt(1 + t^2) by two Newton steps from the FP32 estimate, s = t c,
// so c^2 + s^2 = 1 to FP64 rounding.  An approximate angle leaves a small
// M_PQ behind for the next sweep; the update itself is the full similarity
// J^T M J in FP64, so the eigenvectors keep FP64 accuracy.
template <int P, int Q>
__device__ __forceinline__ void jacobi_rotate(double (&M)[4][4], double (&V)[4][4]) {
    const double apq = M[P][Q];
    if (apq == 0.0) return;
    const float tau = (float)(M[Q][Q] - M[P][P]) / (2.0f * (float)apq);
    const float tf = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
    if (tf == 0.0f) return;  // |M_PQ| negligible against |M_QQ - M_PP|
    const double t = tf;
    const double x = fma(t, t, 1.0);
    double c = (double)rsqrtf((float)x);
    c = c * fma(-0.5 * x, c * c, 1.5);
    c = c * fma(-0.5 * x, c * c, 1.5);
    const double s = t * c;
    const double cc = c * c, ss = s * s, cs = c * s;
    const double app = M[P][P], aqq = M[Q][Q];
    M[P][P] = fma(cc, app, fma(-2.0 * cs, apq, ss * aqq));
    M[Q][Q] = fma(ss, app, fma(2.0 * cs, apq, cc * aqq));
    M[P][Q] = fma(cc - ss, apq, cs * (app - aqq));
#pragma unroll
    for (int k = 0; k < 4; ++k) {  // the other rows / columns of J^T M J
        if (k == P || k == Q) continue;
        double &mkp = k < P ? M[k][P] : M[P][k];
        double &mkq = k < Q ? M[k][Q] : M[Q][k];
        const double a = mkp, b = mkq;
        mkp = fma(c, a, -s * b);
        mkq = fma(s, a, c * b);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {  // eigenvectors accumulate as columns of V J
        const double a = V[k][P], b = V[k][Q];
        V[k][P] = fma(c, a, -s * b);
        V[k][Q] = fma(s, a, c * b);
    }
}

// Homogeneous point X (4) minimising |A X| / |X|, from the 4 rows of A.
__device__ __forceinline__ void dlt_null_vector(const double (&A)[4][4], double (&X)[4]) {
    double M[4][4], V[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            if (j >= i) {  // upper triangle only
#pragma unroll
                for (int r = 0; r < 4; ++r) s += A[r][i] * A[r][j];
            }
            M[i][j] = s;
            V[i][j] = i == j ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        const double off = M[0][1] * M[0][1] + M[0][2] * M[0][2] + M[0][3] * M[0][3] + M[1][2] * M[1][2] +
                           M[1][3] * M[1][3] + M[2][3] * M[2][3];
        const double dia = M[0][0] * M[0][0] + M[1][1] * M[1][1] + M[2][2] * M[2][2] + M[3][3] * M[3][3];
        if (off <= 1e-34 * dia) break;
        jacobi_rotate<0, 1>(M, V);
        jacobi_rotate<0, 2>(M, V);
        jacobi_rotate<0, 3>(M, V);
        jacobi_rotate<1, 2>(M, V);
        jacobi_rotate<1, 3>(M, V);
        jacobi_rotate<2, 3>(M, V);
    }
    // column of the smallest eigenvalue (constant indices only: M and V stay in registers)
    double best = M[0][0];
#pragma unroll
    for (int i = 0; i < 4; ++i) X[i] = V[i][0];
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (M[j][j] < best) {
            best = M[j][j];
#pragma unroll
            for (int i = 0; i < 4; ++i) X[i] = V[i][j];
        }
}

struct GateOut {
    float x, y, z;
    uint8_t status, reason;
};

__device__ __forceinline__ GateOut gate_point(const GateArgs &g, float2 pl, float2 pr, bool tracked) {
    GateOut o{0.f, 0.f, 0.f, 0, VT_LOST_INPUT};
    if (!tracked || !isfinite(pl.x) || !isfinite(pl.y) || !isfinite(pr.x) || !isfinite(pr.y)) return o;
    const double *KL = g.rig.kl, *KR = g.rig.kr, *R = g.rig.R, *T = g.rig.t;
    const double ul = pl.x, vl = pl.y, ur = pr.x, vr = pr.y;
    const double xl = (ul - KL[2]) / KL[0], yl = (vl - KL[3]) / KL[1];
    const double xr = (ur - KR[2]) / KR[0], yr = (vr - KR[3]) / KR[1];
    // disparity against the right image of the left ray's point at infinity
    const double rx = R[0] * xl + R[1] * yl + R[2];
    const double ry = R[3] * xl + R[4] * yl + R[5];
    const double rz = R[6] * xl + R[7] * yl + R[8];
    if (rz > 0.0) {
        const double dx = ur - (KR[0] * rx / rz + KR[2]);
        const double dy = vr - (KR[1] * ry / rz + KR[3]);
        if (!(sqrt(dx * dx + dy * dy) > g.prm.min_disp)) {
            o.reason = VT_LOST_DISP;
            return o;
        }
    }
    // rows x P^3 - P^1 and y P^3 - P^2 of both views
    const double A[4][4] = {{-1.0, 0.0, xl, 0.0},
                            {0.0, -1.0, yl, 0.0},
                            {xr * R[6] - R[0], xr * R[7] - R[1], xr * R[8] - R[2], xr * T[2] - T[0]},
                            {yr * R[6] - R[3], yr * R[7] - R[4], yr * R[8] - R[5], yr * T[2] - T[1]}};
    double Xh[4];
    dlt_null_vector(A, Xh);
    o.reason = VT_LOST_DEPTH;
    if (Xh[3] == 0.0) return o;
    const double X = Xh[0] / Xh[3], Y = Xh[1] / Xh[3], Z = Xh[2] / Xh[3];
    o.x = (float)X;
    o.y = (float)Y;
    o.z = (float)Z;
    const double XR = R[0] * X + R[1] * Y + R[2] * Z + T[0];
    const double YR = R[3] * X + R[4] * Y + R[5] * Z + T[1];
    const double ZR = R[6] * X + R[7] * Y + R[8] * Z + T[2];
    if (!(ZR > 0.0 && Z >= g.prm.z_min && Z <= g.prm.z_max)) return o;
    const double exl = KL[0] * X / Z + KL[2] - ul, eyl = KL[1] * Y / Z + KL[3] - vl;
    const double exr = KR[0] * XR / ZR + KR[2] - ur, eyr = KR[1] * YR / ZR + KR[3] - vr;
    const double el = sqrt(exl * exl + eyl * eyl), er = sqrt(exr * exr + eyr * eyr);
    if (!(fmax(el, er) <= g.prm.max_reproj)) {
        o.reason = VT_LOST_REPROJ;
        return o;
    }
    o.status = 1;
    o.reason = VT_TRACKED;
    return o;
}

__global__ void __launch_bounds__(128) k_stereo_gate(const float2 *pl, const float2 *pr, const uint8_t *st_in, int n,
                                                     GateArgs g, float *xyz, uint8_t *st_out, uint8_t *reason) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const GateOut o = gate_point(g, pl[i], pr[i], st_in ? st_in[i] != 0 : true);
    if (xyz) {
        xyz[3 * i + 0] = o.x;
        xyz[3 * i + 1] = o.y;
        xyz[3 * i + 2] = o.z;
    }
    st_out[i] = o.status;
    if (reason) reason[i] = o.reason;
}

// Batched form: every gate task of a vt_batch table, one thread per pair,
// grid-stride (the grid is fixed so a captured graph replays any batch).
__global__ void __launch_bounds__(128) k_gate_batch(const uint8_t *tab) {
    const BatchHdr *H = reinterpret_cast<const BatchHdr *>(tab);
    const GTask *gates = reinterpret_cast<const GTask *>(tab + H->off_gates);
    const int *p0s = reinterpret_cast<const int *>(tab + H->off_gprefix);
    const int total = H->gate_points, ng = H->ngates;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
        int lo = 0, hi = ng - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(p0s + mid) <= p) lo = mid;
            else hi = mid - 1;
        }
        const GTask &t = gates[lo];
        const int i = p - t.p0;
        GateArgs g;
        g.rig = t.rig;
        g.prm = H->G;
        const GateOut o = gate_point(g, t.pts_l[i], t.pts_r[i], t.status_in ? t.status_in[i] != 0 : true);
        if (t.xyz) {
            t.xyz[3 * i + 0] = o.x;
            t.xyz[3 * i + 1] = o.y;
            t.xyz[3 * i + 2] = o.z;
        }
        t.status_out[i] = o.status;
        if (t.reason) t.reason[i] = o.reason;
    }
}

static bool finite_all(const double *v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

bool gate_args_ok(const vt_stereo_rig *rig, const vt_gate_params *prm) {
    if (!rig || !prm) return false;
    if (!finite_all(rig->kl, 4) || !finite_all(rig->kr, 4) || !finite_all(rig->R, 9) || !finite_all(rig->t, 3))
        return false;
    if (rig->kl[0] == 0.0 || rig->kl[1] == 0.0 || rig->kr[0] == 0.0 || rig->kr[1] == 0.0) return false;
    return prm->min_disp >= 0.0 && prm->max_reproj >= 0.0 && prm->z_min <= prm->z_max && std::isfinite(prm->z_min);
}

vt_status launch_gate_batch(const uint8_t *dev_tab, int grid, cudaStream_t s) {
    k_gate_batch<<<grid, 128, 0, s>>>(dev_tab);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}

}  // namespace vt

using namespace vt;

extern "C" vt_status vt_stereo_gate(const float *pts_l, const float *pts_r, const uint8_t *status_in, int n,
                                    const vt_stereo_rig *rig, const vt_gate_params *prm, float *xyz_out,
                                    uint8_t *status_out, uint8_t *reason_out, void *cuda_stream) {
    if (n < 0 || !gate_args_ok(rig, prm)) return VT_ERR_ARG;
    if (n > 0 && (!pts_l || !pts_r || !status_out)) return VT_ERR_ARG;
    if (n == 0) return VT_OK;
    GateArgs g;
    g.rig = *rig;
    g.prm = *prm;
    const int blocks = (n + 127) / 128;
    k_stereo_gate<<<blocks, 128, 0, (cudaStream_t)cuda_stream>>>(reinterpret_cast<const float2 *>(pts_l),
                                                                 reinterpret_cast<const float2 *>(pts_r), status_in,
                                                                 n, g, xyz_out, status_out, reason_out);
    return cudaGetLastError() == cudaSuccess ? VT_OK : VT_ERR_CUDA;
}
