/*
 * FP64 CPU oracle for the pyramidal Lucas-Kanade (KLT) hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this file's library.  The
 * CUDA library shares no code, header, table or helper with it.
 *
 * What it computes.  The paper uses Shi-Tomasi corners with LK optical-flow
 * tracking as its classical front-end (Sec. IV, citing Lucas-Kanade), the same
 * KLT tracker VINS-Fusion uses (Table I); LK tracking needs keypoints only
 * (Sec. III-A) and, in stereo, only features that pass the cross-camera
 * optical-flow check enter the temporal pool (Sec. V-A).  The paper states
 * none of the algorithm's constants, so every step below follows the textbook
 * coarse-to-fine Lucas-Kanade iteration, with these readings:
 *
 *   pyramid  level l+1 (size ceil(w/2) x ceil(h/2)) is the 25-tap separable
 *            [1 4 6 4 1] x [1 4 6 4 1] / 256 sum centred at (2x, 2y) of level
 *            l, reflect-101 borders (clamp when a side is 1 px), rounded as
 *            (s + 128) >> 8.  Written here as the plain 2-D sum.
 *   gradient Scharr [-3 0 3; -10 0 10; -3 0 3] for d/dx and its transpose for
 *            d/dy, reflect-101 borders, raw integer output; raw / 32 is the
 *            derivative in grey levels per pixel.
 *   coords   pixel centres at integer coordinates; level-l coordinate =
 *            level-0 coordinate / 2^l.
 *   sampling bilinear with replicate-clamped neighbour indices; the template
 *            gradient is the bilinear sample of the stored gradient planes.
 *   LK       per level l = L-1 .. 0 with u_l = u / 2^l and window offsets
 *            x in [-h, h]^2 (h = win / 2):
 *              T(x) = I_l(u_l + x),  grad T(x) = (Ix, Iy)(u_l + x)
 *              G = sum [Ix^2, Ix Iy; Ix Iy, Iy^2]
 *              reject if lambda_min(G) / (win^2 255^2) < min_eig or det <= 0
 *              nu = 0; for k < max_iters:
 *                 q = u_l + g_l + nu, reject if q leaves
 *                     [-h, w_l - 1 + h] x [-h, h_l - 1 + h]
 *                 r(x) = T(x) - J_l(q + x),  b = sum r (Ix, Iy)
 *                 eta = G^-1 b, nu += eta, stop if |eta|^2 < eps^2
 *              g_{l-1} = 2 (g_l + nu)
 *            result v = u + g_0 + nu; reject if v leaves [0, W-1] x [0, H-1];
 *            error = mean |T(x) - J_0(v + x)| over the window.
 *            Initial g_{L-1} = 0, or (guess - u) / 2^(L-1) when a guess is given.
 *   FB       ok = status_fwd & status_bwd & |p - back(fwd(p))|_2 <= thr.
 *
 * Per point it also reports, for each kind of threshold decision, the
 * smallest margin by which that decision was taken (relative for the
 * eigenvalue test, in pixels otherwise), so that a status disagreement with a
 * single-precision implementation can be attributed to the decision that
 * produced it being taken within 1e-4 of its threshold: the eigenvalue test
 * at every level examined, the image-bound test at every evaluation, and the
 * convergence test both over every iteration and at the deciding iterations
 * only (those that stopped a level's loop).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_LOST_EIG = 1, ORC_LOST_OOB = 2, ORC_LOST_FB = 3, ORC_LOST_INPUT = 4 };

/* Reflect-101 border index (..., 2, 1 | 0, 1, 2, ..., n-1 | n-2, ...); a 1-px
 * side has nothing to reflect, so it clamps. */
static int refl101(int i, int n)
{
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * n - 2 - i;
    }
    return i;
}

static int clampi(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

/* One Gaussian-pyramid step: dst = pyrDown(src). */
void orc_pyrdown(const uint8_t *src, int w, int h, int spitch, uint8_t *dst, int dpitch)
{
    static const int k[5] = {1, 4, 6, 4, 1};
    const int W = (w + 1) / 2, H = (h + 1) / 2;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long s = 0;
            for (int j = 0; j < 5; ++j)
                for (int i = 0; i < 5; ++i) {
                    int sy = refl101(2 * y + j - 2, h);
                    int sx = refl101(2 * x + i - 2, w);
                    s += (long)(k[i] * k[j]) * src[(long)sy * spitch + sx];
                }
            dst[(long)y * dpitch + x] = (uint8_t)((s + 128) >> 8);
        }
}

/* Scharr derivatives, raw integer output in [-4080, 4080]. */
void orc_scharr(const uint8_t *src, int w, int h, int spitch, int16_t *gx, int16_t *gy, int gpitch)
{
    static const int smooth[3] = {3, 10, 3};
    static const int diff[3] = {-1, 0, 1};
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int sx = 0, sy = 0;
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i) {
                    int v = src[(long)refl101(y + j, h) * spitch + refl101(x + i, w)];
                    sx += smooth[j + 1] * diff[i + 1] * v;
                    sy += smooth[i + 1] * diff[j + 1] * v;
                }
            gx[(long)y * gpitch + x] = (int16_t)sx;
            gy[(long)y * gpitch + x] = (int16_t)sy;
        }
}

/* One pyramid level in double precision, tight row-major (pitch = w). */
typedef struct {
    const double *img; /* grey levels */
    const double *gx;  /* d img / dx, grey levels per pixel (may be NULL for J) */
    const double *gy;
    int w, h;
} orc_level;

typedef struct {
    int win;       /* odd window side */
    int levels;    /* levels used, <= levels of both pyramids */
    int max_iters; /* Newton iterations per level */
    double eps;    /* convergence threshold on |eta| in level pixels */
    double min_eig;/* threshold on lambda_min(G) / (win^2 255^2) */
} orc_params;

static double bilinear(const double *a, int w, int h, double x, double y)
{
    const double fx = floor(x), fy = floor(y);
    const int x0 = (int)fx, y0 = (int)fy;
    const double ax = x - fx, ay = y - fy;
    const int xa = clampi(x0, 0, w - 1), xb = clampi(x0 + 1, 0, w - 1);
    const int ya = clampi(y0, 0, h - 1), yb = clampi(y0 + 1, 0, h - 1);
    return (1.0 - ax) * (1.0 - ay) * a[(long)ya * w + xa] + ax * (1.0 - ay) * a[(long)ya * w + xb] +
           (1.0 - ax) * ay * a[(long)yb * w + xa] + ax * ay * a[(long)yb * w + xb];
}

static double dmin(double a, double b) { return a < b ? a : b; }

/*
 * Track n points from pyramid I to pyramid J.
 *   pts     [n][2] level-0 (x, y) in I
 *   guess   [n][2] level-0 guess in J, or NULL
 *   out     [n][2] tracked position in J (last estimate when lost)
 *   status  [n]    1 tracked, 0 lost
 *   err     [n]    mean |T - J| at level 0 (0 when lost)
 *   reason  [n]    ORC_* code
 *   iters   [n]    Newton iterations summed over levels
 *   iters_level [n][levels] (may be NULL) Newton iterations at each level
 *   lmin    [n]    normalised lambda_min of G at the last level examined
 *   margin  [n][4] smallest |lambda_min - min_eig| / min_eig over the levels
 *                  examined; smallest | |eta| - eps | over every iteration;
 *                  smallest distance to the image-bound tests; smallest
 *                  | |eta| - eps | at the iterations that stopped a level
 */
void orc_track(const orc_level *I, const orc_level *J, const orc_params *prm, const double *pts,
               const double *guess, int n, double *out, uint8_t *status, double *err, uint8_t *reason,
               int32_t *iters, double *lmin, double *margin, int32_t *iters_level)
{
    const int win = prm->win, hw = win / 2, N = win * win, L = prm->levels;
    double *T = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *TX = T + N, *TY = T + 2 * N;
    for (int p = 0; p < n; ++p) {
        const double ux0 = pts[2 * p], uy0 = pts[2 * p + 1];
        double m_eig = INFINITY, m_conv = INFINITY, m_bnd = INFINITY, m_stop = INFINITY, lm = NAN;
        int st = 1, rs = ORC_OK, it = 0;
        double gx = 0.0, gy = 0.0, nux = 0.0, nuy = 0.0;
        double ex = 0.0, ey = 0.0;
        int lost_level = -1;
        if (iters_level)
            for (int l = 0; l < L; ++l) iters_level[(size_t)p * L + l] = 0;
        if (!(ux0 >= 0.0 && ux0 <= I[0].w - 1 && uy0 >= 0.0 && uy0 <= I[0].h - 1)) {
            st = 0;
            rs = ORC_LOST_INPUT;
            lost_level = 0;
            goto done;
        }
        if (guess) {
            const double s = ldexp(1.0, -(L - 1));
            gx = (guess[2 * p] - ux0) * s;
            gy = (guess[2 * p + 1] - uy0) * s;
        }
        for (int l = L - 1; l >= 0; --l) {
            const orc_level *Il = &I[l], *Jl = &J[l];
            const double s = ldexp(1.0, -l);
            const double ux = ux0 * s, uy = uy0 * s;
            double g11 = 0.0, g12 = 0.0, g22 = 0.0;
            for (int j = 0; j < win; ++j)
                for (int i = 0; i < win; ++i) {
                    const double x = ux + (i - hw), y = uy + (j - hw);
                    const int k = j * win + i;
                    T[k] = bilinear(Il->img, Il->w, Il->h, x, y);
                    TX[k] = bilinear(Il->gx, Il->w, Il->h, x, y);
                    TY[k] = bilinear(Il->gy, Il->w, Il->h, x, y);
                    g11 += TX[k] * TX[k];
                    g12 += TX[k] * TY[k];
                    g22 += TY[k] * TY[k];
                }
            lm = (g11 + g22 - sqrt((g11 - g22) * (g11 - g22) + 4.0 * g12 * g12)) * 0.5 /
                 ((double)N * 255.0 * 255.0);
            m_eig = dmin(m_eig, fabs(lm - prm->min_eig) / prm->min_eig);
            const double det = g11 * g22 - g12 * g12;
            if (!(lm >= prm->min_eig) || !(det > 0.0)) {
                st = 0;
                rs = ORC_LOST_EIG;
                lost_level = l;
                nux = nuy = 0.0;
                goto done;
            }
            nux = nuy = 0.0;
            for (int k = 0; k < prm->max_iters; ++k) {
                const double qx = ux + gx + nux, qy = uy + gy + nuy;
                const double dist = dmin(dmin(qx + hw, (Jl->w - 1 + hw) - qx), dmin(qy + hw, (Jl->h - 1 + hw) - qy));
                m_bnd = dmin(m_bnd, fabs(dist));
                if (!(dist >= 0.0)) {
                    st = 0;
                    rs = ORC_LOST_OOB;
                    lost_level = l;
                    goto done;
                }
                double b1 = 0.0, b2 = 0.0;
                for (int j = 0; j < win; ++j)
                    for (int i = 0; i < win; ++i) {
                        const int kk = j * win + i;
                        const double r = T[kk] - bilinear(Jl->img, Jl->w, Jl->h, qx + (i - hw), qy + (j - hw));
                        b1 += r * TX[kk];
                        b2 += r * TY[kk];
                    }
                ex = (g22 * b1 - g12 * b2) / det;
                ey = (g11 * b2 - g12 * b1) / det;
                nux += ex;
                nuy += ey;
                ++it;
                if (iters_level) ++iters_level[(size_t)p * L + l];
                const double step = fabs(sqrt(ex * ex + ey * ey) - prm->eps);
                m_conv = dmin(m_conv, step);
                if (ex * ex + ey * ey < prm->eps * prm->eps) {
                    m_stop = dmin(m_stop, step);
                    break;
                }
            }
            if (l > 0) {
                gx = 2.0 * (gx + nux);
                gy = 2.0 * (gy + nuy);
            }
        }
        lost_level = 0;
    done:;
        /* position: level-0 estimate; when lost at level l, the level-l
         * estimate scaled back to level 0 */
        {
            const double s = ldexp(1.0, lost_level < 0 ? 0 : lost_level);
            const double ux = ux0 / s, uy = uy0 / s;
            out[2 * p] = (ux + gx + nux) * s;
            out[2 * p + 1] = (uy + gy + nuy) * s;
        }
        double e = 0.0;
        if (st) {
            const double vx = out[2 * p], vy = out[2 * p + 1];
            const double dist = dmin(dmin(vx, (I[0].w - 1) - vx), dmin(vy, (I[0].h - 1) - vy));
            m_bnd = dmin(m_bnd, fabs(dist));
            if (!(dist >= 0.0)) {
                st = 0;
                rs = ORC_LOST_OOB;
            } else {
                for (int j = 0; j < win; ++j)
                    for (int i = 0; i < win; ++i) {
                        const int kk = j * win + i;
                        e += fabs(T[kk] - bilinear(J[0].img, J[0].w, J[0].h, vx + (i - hw), vy + (j - hw)));
                    }
                e /= (double)N;
            }
        }
        status[p] = (uint8_t)st;
        reason[p] = (uint8_t)rs;
        err[p] = st ? e : 0.0;
        iters[p] = it;
        lmin[p] = lm;
        margin[4 * p] = m_eig;
        margin[4 * p + 1] = m_conv;
        margin[4 * p + 2] = m_bnd;
        margin[4 * p + 3] = m_stop;
    }
    free(T);
}

/* Forward-backward consistency: ok = st_f & st_b & |p0 - p0_back|_2 <= thr. */
void orc_fb_check(const double *p0, const double *p0b, const uint8_t *st_f, const uint8_t *st_b, int n,
                  double thr, uint8_t *status, double *dist, double *margin)
{
    for (int i = 0; i < n; ++i) {
        const double dx = p0[2 * i] - p0b[2 * i], dy = p0[2 * i + 1] - p0b[2 * i + 1];
        const double d = sqrt(dx * dx + dy * dy);
        dist[i] = d;
        margin[i] = fabs(d - thr);
        status[i] = (uint8_t)(st_f[i] && st_b[i] && d <= thr);
    }
}

/*
 * Shi-Tomasi (GFTT) corner detection: the paper's classical front-end pairs
 * Shi-Tomasi corners with LK tracking (Sec. IV) and runs it on the CPU
 * (Sec. V-F).  Reading implemented (the paper gives no parameters):
 *   gradients   raw Scharr int16 of the level (gx, gy);
 *   tensor      a = sum gx^2, b = sum gx gy, c = sum gy^2 over the
 *               (2 br + 1)^2 block around the pixel, reflect-101 borders,
 *               exact integers;
 *   score       lambda = ((a + c) - sqrt((a - c)^2 + 4 b^2)) / 2 evaluated in
 *               single precision, operation by operation (so that every
 *               decision below is the same as the CUDA kernel's), clamped
 *               at 0;
 *   candidate   lambda >= quality * max(lambda) and lambda > 0, at least
 *               `border` px from every image edge, a local maximum of its
 *               (2 nms + 1)^2 neighbourhood (ties: the smaller row-major
 *               index wins), and at squared distance >= min_dist^2 from
 *               every mask point (points already tracked);
 *   selection   candidates in priority order (lambda descending, index
 *               ascending); a candidate is kept when no kept corner lies at
 *               squared distance < min_dist^2; at most max_corners are kept.
 * Output: kept corners in priority order (x, y integers) and their scores.
 */
float orc_gftt_score(long a, long b, long c)
{
    const float fa = (float)a, fb = (float)b, fc = (float)c;
    const volatile float d = fa - fc;
    const volatile float d2 = d * d;
    const volatile float b2 = fb * fb;
    const volatile float b4 = 4.0f * b2;
    const volatile float q = d2 + b4;
    const volatile float r = sqrtf(q);
    const volatile float s = fa + fc;
    const volatile float t = s - r;
    const float l = 0.5f * t;
    return l > 0.0f ? l : 0.0f;
}

int orc_gftt(const int16_t *gx, const int16_t *gy, int w, int h, int gpitch, int br, float quality, int nms,
             int border, int min_dist, const double *mask, int n_mask, int max_corners, int32_t *out_xy,
             float *out_score)
{
    float *score = (float *)malloc(sizeof(float) * (size_t)w * h);
    float mx = 0.0f;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            long a = 0, b = 0, c = 0;
            for (int j = -br; j <= br; ++j)
                for (int i = -br; i <= br; ++i) {
                    const long o = (long)refl101(y + j, h) * gpitch + refl101(x + i, w);
                    const long u = gx[o], v = gy[o];
                    a += u * u;
                    b += u * v;
                    c += v * v;
                }
            const float s = orc_gftt_score(a, b, c);
            score[(long)y * w + x] = s;
            if (s > mx) mx = s;
        }
    const volatile float thr = quality * mx;
    /* candidates */
    long cap = 1024, n = 0;
    long *cand = (long *)malloc(sizeof(long) * cap);
    for (int y = border; y < h - border; ++y)
        for (int x = border; x < w - border; ++x) {
            const long idx = (long)y * w + x;
            const float s = score[idx];
            if (!(s >= thr) || !(s > 0.0f)) continue;
            int ok = 1;
            for (int j = -nms; j <= nms && ok; ++j)
                for (int i = -nms; i <= nms; ++i) {
                    const int yy = y + j, xx = x + i;
                    if ((i == 0 && j == 0) || yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                    const long q = (long)yy * w + xx;
                    const float t = score[q];
                    if (t > s || (t == s && q < idx)) {
                        ok = 0;
                        break;
                    }
                }
            for (int m = 0; m < n_mask && ok; ++m) {
                const volatile float dx = (float)x - (float)mask[2 * m];
                const volatile float dy = (float)y - (float)mask[2 * m + 1];
                const volatile float dd = dx * dx + dy * dy;
                if (dd < (float)(min_dist * min_dist)) ok = 0;
            }
            if (!ok) continue;
            if (n == cap) {
                cap *= 2;
                cand = (long *)realloc(cand, sizeof(long) * cap);
            }
            cand[n++] = idx;
        }
    /* priority order: score descending, index ascending (insertion into a
     * sorted array is plain and obviously right; n is small) */
    for (long i = 1; i < n; ++i) {
        const long v = cand[i];
        long j = i - 1;
        while (j >= 0) {
            const long u = cand[j];
            const int before = score[v] > score[u] || (score[v] == score[u] && v < u);
            if (!before) break;
            cand[j + 1] = u;
            --j;
        }
        cand[j + 1] = v;
    }
    int kept = 0;
    for (long i = 0; i < n && kept < max_corners; ++i) {
        const int x = (int)(cand[i] % w), y = (int)(cand[i] / w);
        int ok = 1;
        for (int k = 0; k < kept; ++k) {
            const long dx = x - out_xy[2 * k], dy = y - out_xy[2 * k + 1];
            if (dx * dx + dy * dy < (long)min_dist * min_dist) {
                ok = 0;
                break;
            }
        }
        if (!ok) continue;
        out_xy[2 * kept] = x;
        out_xy[2 * kept + 1] = y;
        out_score[kept] = score[cand[i]];
        ++kept;
    }
    free(cand);
    free(score);
    return kept;
}
