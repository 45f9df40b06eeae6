"""Coherence-enhancing diffusion tensor, FP64 numpy (TEST INFRASTRUCTURE).

Follows Sec. 4.4 (Eq. parabolique and the definitions after it):
u_sigma = K_sigma * u, J_rho = K_rho * (grad u_sigma grad u_sigma^T); D(J_rho)
has the eigenvectors (v1, v2) of J_rho; with eigenvalues mu1 >= mu2 of J_rho,
D's eigenvalues are lambda1 = alpha (along v1) and
lambda2 = alpha + (1 - alpha) exp(-C / (mu1 - mu2)^2) (along v2).

Readings where the paper is silent:
* sigma and rho are the standard deviations of the Gaussians; the kernel is
  truncated at radius int(3 s + 0.5) and normalised to unit sum;
* every convolution and the gradient reflect the image about its border
  (half-sample symmetric: u(-1) = u(0));
* the gradient is the centred difference (u(i+1) - u(i-1)) / 2;
* exp(-C / 0) = 0, so where mu1 == mu2 the tensor is alpha * I.
"""
import numpy as np


def gaussian_taps(s):
    r = int(3.0 * s + 0.5)
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * k * k / (s * s))
    return w / w.sum()


def blur1d(a, s, axis):
    w = gaussian_taps(s)
    r = (len(w) - 1) // 2
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    ap = np.pad(a, pad, mode="symmetric")
    n = a.shape[axis]
    out = np.zeros_like(a, dtype=np.float64)
    for j, wj in enumerate(w):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(j, j + n)
        out += wj * ap[tuple(sl)]
    return out


def blur(a, s):
    """Separable Gaussian of standard deviation s over the last two axes."""
    return blur1d(blur1d(np.asarray(a, np.float64), s, -1), s, -2)


def gradient(a):
    """Centred differences with a reflected border; returns (gx, gy)."""
    ap = np.pad(np.asarray(a, np.float64), ((1, 1), (1, 1)), mode="symmetric")
    gx = 0.5 * (ap[1:-1, 2:] - ap[1:-1, :-2])
    gy = 0.5 * (ap[2:, 1:-1] - ap[:-2, 1:-1])
    return gx, gy


def structure_tensor(u, sigma, rho):
    us = blur(u, sigma)
    gx, gy = gradient(us)
    return blur(gx * gx, rho), blur(gx * gy, rho), blur(gy * gy, rho)


def tensor_from_J(Jxx, Jxy, Jyy, alpha, C):
    """D(J): same eigenvectors as J; lambda1 = alpha on v1 (eigenvalue mu1 >=
    mu2), lambda2 = alpha + (1 - alpha) exp(-C / (mu1 - mu2)^2) on v2.
    Written with the closed-form 2x2 eigen-decomposition:
    mu1 - mu2 = sqrt((Jxx - Jyy)^2 + 4 Jxy^2), v1 v1^T = (I + R) / 2 with
    R = [[cos 2t, sin 2t], [sin 2t, -cos 2t]], cos 2t = (Jxx - Jyy)/(mu1 - mu2),
    sin 2t = 2 Jxy / (mu1 - mu2)."""
    Jxx, Jxy, Jyy = (np.asarray(a, np.float64) for a in (Jxx, Jxy, Jyy))
    delta = np.sqrt((Jxx - Jyy) ** 2 + 4.0 * Jxy ** 2)
    pos = delta > 0
    safe = np.where(pos, delta, 1.0)
    lam1 = np.full_like(delta, alpha)
    lam2 = np.where(pos, alpha + (1.0 - alpha) * np.exp(-C / (safe * safe)), alpha)
    c2 = np.where(pos, (Jxx - Jyy) / safe, 0.0)
    s2 = np.where(pos, 2.0 * Jxy / safe, 0.0)
    m = 0.5 * (lam1 + lam2)
    h = 0.5 * (lam1 - lam2)
    return m + h * c2, h * s2, m - h * c2


def ced_tensor(u, sigma, rho, alpha, C):
    """The full tensor stage (i) of Sec. 4.4: returns (Dxx, Dxy, Dyy)."""
    return tensor_from_J(*structure_tensor(u, sigma, rho), alpha, C)
