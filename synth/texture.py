"""Continuous band-limited texture: Gaussian blobs plus sinusoids.

Tex(X, Y) = base + sum_b A_b exp(-((X-cx_b)^2 + (Y-cy_b)^2) / (2 s_b^2))
                 + sum_s a_s sin(kx_s X + ky_s Y + phi_s)

The texture is evaluated exactly (no resampling) on an affine image of the
pixel grid, so a second frame related to the first by a known rotation and
translation has a closed-form ground-truth flow.

Defaults follow the workload recipe: 400 blobs with centres uniform over the
image extended by a margin, sigma ~ U[2, 12] px, amplitude ~ U[-80, 80] on a
base of 128, plus 64 sinusoids of wavelength >= 8 px with random direction and
phase, wavelength ~ U[8, 32] px and equal amplitudes 20 sqrt(2/64), so that
the noise sum has an RMS of 20 grey levels.  Frames are
clipped to [0, 255] and rounded to the nearest integer.
"""

from __future__ import annotations

import numpy as np

# Blobs are evaluated over a window of +-BLOB_RADIUS_SIGMAS sigma; beyond it a
# blob of amplitude 80 contributes < 80 * exp(-12.5) ~ 3e-4 grey levels.
BLOB_RADIUS_SIGMAS = 5.0


def affine_from_motion(theta_deg: float, tx: float, ty: float, cx: float, cy: float) -> np.ndarray:
    """2x3 matrix of the rigid motion p -> R(theta) (p - c) + c + t."""
    th = np.deg2rad(theta_deg)
    c, s = np.cos(th), np.sin(th)
    R = np.array([[c, -s], [s, c]])
    cvec = np.array([cx, cy])
    off = cvec + np.array([tx, ty]) - R @ cvec
    return np.hstack([R, off[:, None]])


def invert_affine(A: np.ndarray) -> np.ndarray:
    M = A[:, :2]
    Mi = np.linalg.inv(M)
    return np.hstack([Mi, (-Mi @ A[:, 2])[:, None]])


class BlobTexture:
    """Seeded texture on the plane.  Coordinates are in texture pixels."""

    def __init__(
        self,
        seed: int,
        extent: tuple[float, float, float, float],
        n_blobs: int = 400,
        sigma_range: tuple[float, float] = (2.0, 12.0),
        amp_range: tuple[float, float] = (-80.0, 80.0),
        base: float = 128.0,
        n_sin: int = 64,
        wavelength_range: tuple[float, float] = (8.0, 32.0),
        noise_amp: float = 20.0,
        blob_radius_sigmas: float = BLOB_RADIUS_SIGMAS,
    ):
        rng = np.random.Generator(np.random.PCG64(seed))
        x0, y0, x1, y1 = extent
        self.base = float(base)
        self.blob_radius_sigmas = float(blob_radius_sigmas)
        self.cx = rng.uniform(x0, x1, n_blobs)
        self.cy = rng.uniform(y0, y1, n_blobs)
        self.sig = rng.uniform(sigma_range[0], sigma_range[1], n_blobs)
        self.amp = rng.uniform(amp_range[0], amp_range[1], n_blobs)
        lam = rng.uniform(wavelength_range[0], wavelength_range[1], n_sin)
        ang = rng.uniform(0.0, 2.0 * np.pi, n_sin)
        k = 2.0 * np.pi / lam
        self.kx = k * np.cos(ang)
        self.ky = k * np.sin(ang)
        self.phi = rng.uniform(0.0, 2.0 * np.pi, n_sin)
        self.a = np.full(n_sin, noise_amp * np.sqrt(2.0 / max(n_sin, 1)))

    # ------------------------------------------------------------------ eval
    def eval_affine(self, w: int, h: int, A: np.ndarray, with_grad: bool = False):
        """Evaluate on pixel (x, y), x<w, y<h, mapped to texture coords A @ [x, y, 1].

        Returns float64 [h, w] (and, with ``with_grad``, the exact derivatives
        with respect to the pixel coordinates x and y)."""
        A = np.asarray(A, dtype=np.float64)
        out = np.full((h, w), self.base, dtype=np.float64)
        gx = np.zeros((h, w)) if with_grad else None
        gy = np.zeros((h, w)) if with_grad else None
        self._add_sinusoids(out, gx, gy, A)
        self._add_blobs(out, gx, gy, A)
        if with_grad:
            return out, gx, gy
        return out

    def _add_sinusoids(self, out, gx, gy, A):
        h, w = out.shape
        # phase_s(x, y) = al_s x + be_s y + ga_s
        al = self.kx * A[0, 0] + self.ky * A[1, 0]
        be = self.kx * A[0, 1] + self.ky * A[1, 1]
        ga = self.kx * A[0, 2] + self.ky * A[1, 2] + self.phi
        xs = np.arange(w, dtype=np.float64)
        ys = np.arange(h, dtype=np.float64)
        px = np.outer(xs, al)  # [w, S]
        py = np.outer(ys, be) + ga  # [h, S]
        sx, cxv = np.sin(px), np.cos(px)
        sy, cyv = np.sin(py), np.cos(py)
        a = self.a
        # sin(u + v) = sin u cos v + cos u sin v
        out += (cyv * a) @ sx.T + (sy * a) @ cxv.T
        if gx is not None:
            # d/dx sin(al x + be y + ga) = al cos(...), cos(u+v) = cos u cos v - sin u sin v
            gx += (cyv * (a * al)) @ cxv.T - (sy * (a * al)) @ sx.T
            gy += (cyv * (a * be)) @ cxv.T - (sy * (a * be)) @ sx.T

    def _add_blobs(self, out, gx, gy, A):
        h, w = out.shape
        Ai = invert_affine(A)
        M = A[:, :2]
        # pixel-space extent of a texture-space disc of radius r: r * ||Ai rows||
        sx_scale = np.hypot(Ai[0, 0], Ai[0, 1])
        sy_scale = np.hypot(Ai[1, 0], Ai[1, 1])
        for cx, cy, s, amp in zip(self.cx, self.cy, self.sig, self.amp):
            r = self.blob_radius_sigmas * s
            pxc = Ai[0, 0] * cx + Ai[0, 1] * cy + Ai[0, 2]
            pyc = Ai[1, 0] * cx + Ai[1, 1] * cy + Ai[1, 2]
            rx, ry = r * sx_scale + 1.0, r * sy_scale + 1.0
            xa, xb = max(int(np.floor(pxc - rx)), 0), min(int(np.ceil(pxc + rx)), w - 1)
            ya, yb = max(int(np.floor(pyc - ry)), 0), min(int(np.ceil(pyc + ry)), h - 1)
            if xa > xb or ya > yb:
                continue
            xs = np.arange(xa, xb + 1, dtype=np.float64)
            ys = np.arange(ya, yb + 1, dtype=np.float64)[:, None]
            X = A[0, 0] * xs + A[0, 1] * ys + A[0, 2] - cx
            Y = A[1, 0] * xs + A[1, 1] * ys + A[1, 2] - cy
            inv2s2 = 1.0 / (2.0 * s * s)
            g = amp * np.exp(-(X * X + Y * Y) * inv2s2)
            out[ya : yb + 1, xa : xb + 1] += g
            if gx is not None:
                dX = -2.0 * inv2s2 * X * g
                dY = -2.0 * inv2s2 * Y * g
                gx[ya : yb + 1, xa : xb + 1] += dX * M[0, 0] + dY * M[1, 0]
                gy[ya : yb + 1, xa : xb + 1] += dX * M[0, 1] + dY * M[1, 1]

    def eval_points(self, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        """Exact evaluation at scattered texture coordinates (small inputs only)."""
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        out = np.full(X.shape, self.base)
        for k in range(len(self.kx)):
            out += self.a[k] * np.sin(self.kx[k] * X + self.ky[k] * Y + self.phi[k])
        for cx, cy, s, amp in zip(self.cx, self.cy, self.sig, self.amp):
            out += amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * s * s))
        return out


def quantize_u8(img: np.ndarray) -> np.ndarray:
    """Clip to [0, 255] and round to nearest (ties to even)."""
    return np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8)
