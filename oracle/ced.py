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


# ---------------------------------------------------------------- 3D (Sec. 5, 3D experiments)
# The 3D coherence-enhancing tensor: u_sigma, J_rho as above over three axes
# (six channels xx, yy, zz, xy, xz, yz); D(J) has the eigenvectors of J and,
# for eigenvalues mu1 >= mu2 >= mu3 of J, the eigenvalues
# lambda1 = alpha, lambda2 = alpha + (1 - alpha) exp(-C / (mu1 - mu2)^2),
# lambda3 = alpha + (1 - alpha) exp(-C / (mu1 - mu3)^2)   (exp(-C/0) = 0).
# Arrays are indexed [z, y, x]; D is returned as the planes
# (Dxx, Dyy, Dzz, Dxy, Dxz, Dyz) of the 3D stencil construction.

def blur3(a, s):
    """Separable Gaussian of standard deviation s over the three axes (x, y, z)."""
    return blur1d(blur1d(blur1d(np.asarray(a, np.float64), s, -1), s, -2), s, -3)


def gradient3(a):
    """Centred differences with a reflected border; returns (gx, gy, gz)."""
    ap = np.pad(np.asarray(a, np.float64), 1, mode="symmetric")
    gx = 0.5 * (ap[1:-1, 1:-1, 2:] - ap[1:-1, 1:-1, :-2])
    gy = 0.5 * (ap[1:-1, 2:, 1:-1] - ap[1:-1, :-2, 1:-1])
    gz = 0.5 * (ap[2:, 1:-1, 1:-1] - ap[:-2, 1:-1, 1:-1])
    return gx, gy, gz


def structure_tensor3(u, sigma, rho):
    """(Jxx, Jyy, Jzz, Jxy, Jxz, Jyz)."""
    gx, gy, gz = gradient3(blur3(u, sigma))
    return tuple(blur3(p, rho) for p in (gx * gx, gy * gy, gz * gz, gx * gy, gx * gz, gy * gz))


def tensor_from_J3(J, alpha, C):
    """D(J) from the eigen-decomposition of J (numpy's symmetric solver)."""
    Jxx, Jyy, Jzz, Jxy, Jxz, Jyz = (np.asarray(a, np.float64) for a in J)
    M = np.stack([np.stack([Jxx, Jxy, Jxz], -1), np.stack([Jxy, Jyy, Jyz], -1),
                  np.stack([Jxz, Jyz, Jzz], -1)], -2)
    mu, V = np.linalg.eigh(M)                      # ascending: mu[..., 2] = mu1
    d12 = mu[..., 2] - mu[..., 1]
    d13 = mu[..., 2] - mu[..., 0]

    def lam(d):
        pos = d > 0
        return np.where(pos, alpha + (1.0 - alpha) * np.exp(-C / np.where(pos, d * d, 1.0)), alpha)

    L = np.stack([lam(d13), lam(d12), np.full_like(d12, alpha)], -1)   # on v3, v2, v1
    D = np.einsum("...ik,...k,...jk->...ij", V, L, V)
    return D[..., 0, 0], D[..., 1, 1], D[..., 2, 2], D[..., 0, 1], D[..., 0, 2], D[..., 1, 2]


def ced_tensor3(u, sigma, rho, alpha, C):
    return np.stack(tensor_from_J3(structure_tensor3(u, sigma, rho), alpha, C))


# Edge-enhancing diffusion in 3D (Sec. 5, the 3D MRI experiment): the same
# J_rho and eigenvectors v1, v2, v3 (eigenvalues mu1 >= mu2 >= mu3); D's
# eigenvalues are lambda1 = 1 - exp(-C / mu1^2) on v1, lambda2 = 1 -
# exp(-C / mu2^2) on v2 and lambda3 = 1 on v3.  Readings: exp(-C / 0) = 0
# (lambda = 1 where mu = 0, as in the CED definition), and 1 - exp(-x) is
# evaluated as -expm1(-x), its value without cancellation for small x.

def tensor_from_J3_eed(J, C):
    """D(J) of edge-enhancing diffusion (numpy's symmetric eigensolver)."""
    Jxx, Jyy, Jzz, Jxy, Jxz, Jyz = (np.asarray(a, np.float64) for a in J)
    M = np.stack([np.stack([Jxx, Jxy, Jxz], -1), np.stack([Jxy, Jyy, Jyz], -1),
                  np.stack([Jxz, Jyz, Jzz], -1)], -2)
    mu, V = np.linalg.eigh(M)                      # ascending: mu[..., 2] = mu1

    def lam(m):
        q = m * m
        pos = q > 0
        return np.where(pos, -np.expm1(-C / np.where(pos, q, 1.0)), 1.0)

    L = np.stack([np.ones_like(mu[..., 0]), lam(mu[..., 1]), lam(mu[..., 2])], -1)   # on v3, v2, v1
    D = np.einsum("...ik,...k,...jk->...ij", V, L, V)
    return D[..., 0, 0], D[..., 1, 1], D[..., 2, 2], D[..., 0, 1], D[..., 0, 2], D[..., 1, 2]


def eed_tensor3(u, sigma, rho, C):
    return np.stack(tensor_from_J3_eed(structure_tensor3(u, sigma, rho), C))
