"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds none of the method's arithmetic: it only draws diffusion
tensor fields, images and initial states on the host (FP64 numpy, seeded
numpy ``Generator``s) so that the CUDA path and the FP64 oracle can be fed the
same values.  The paper's own inputs (a 512^2 fingerprint photograph, an MRI
volume) are not available; these fields take their shapes and parameter
ranges instead.

Array convention: 2D arrays are (ny, nx), 3D arrays (nz, ny, nx), x fastest.
2D tensor fields are returned as a (3, ny, nx) array of planes (Dxx, Dxy, Dyy);
3D fields as (6, nz, ny, nx) planes (xx, yy, zz, xy, xz, yz).
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def u_uniform(shape, seed):
    """u0 ~ U[0, 1), i.i.d. per grid point."""
    return rng(seed).random(shape)


def D_from_angle(theta, kappa):
    """D = R(theta) diag(1, kappa^-2) R(theta)^T (the constant test tensor of
    Sec. 4.1 when theta = pi/6), broadcast over arrays."""
    c, s = np.cos(theta), np.sin(theta)
    lam2 = 1.0 / np.asarray(kappa, np.float64) ** 2
    Dxx = c * c + lam2 * s * s
    Dxy = (1.0 - lam2) * c * s
    Dyy = s * s + lam2 * c * c
    return np.stack(np.broadcast_arrays(Dxx, Dxy, Dyy))


def spiral_field(n, kappa=10.0):
    """64x64-style spiral field: theta(x, y) = atan2(y - c, x - c) + pi/2 +
    2 pi r / 32 with c = (n - 1)/2 and r the distance to the centre."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    cc = (n - 1) / 2.0
    r = np.hypot(x - cc, y - cc)
    theta = np.arctan2(y - cc, x - cc) + np.pi / 2 + 2 * np.pi * r / 32.0
    return D_from_angle(theta, kappa)


def fingerprint(n, seed, n_waves=8, period=(6.0, 12.0), noise=0.2):
    """Fingerprint-like image: sum of ``n_waves`` plane sinusoids with uniform
    random orientation, period ~ U[6, 12] px and phase ~ U[0, 2 pi), rescaled
    to [0, 1], plus N(0, noise^2) per pixel."""
    g = rng(seed)
    ang = g.uniform(0, np.pi, n_waves)
    per = g.uniform(period[0], period[1], n_waves)
    phi = g.uniform(0, 2 * np.pi, n_waves)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    img = np.zeros((n, n))
    for k in range(n_waves):
        img += np.sin(2 * np.pi * (np.cos(ang[k]) * x + np.sin(ang[k]) * y) / per[k] + phi[k])
    img = (img - img.min()) / (img.max() - img.min())
    return img + g.normal(0.0, noise, img.shape)


def _lattice_coords(n, m):
    """Grid index -> (cell index, fraction) on an m-point lattice spanning n points."""
    t = np.arange(n, dtype=np.float64) * (m - 1) / max(n - 1, 1)
    i0 = np.minimum(np.floor(t).astype(np.int64), m - 2)
    return i0, t - i0


def needle_field3d(n, seed, kappa=20.0, lattice=16, dtype=np.float64):
    """3D SPD field with eigenvalues (1, kappa^-2, kappa^-2) and smooth random
    orientation: seeded random unit vectors v on a lattice^3 grid, the
    projector P = v v^T trilinearly interpolated entrywise, and
    D = eps I + (1 - eps) P with eps = kappa^-2 (SPD, anisotropy <= kappa).
    Returns the six planes (Dxx, Dyy, Dzz, Dxy, Dxz, Dyz), each (n, n, n),
    computed one z plane at a time (FP64, then cast to dtype)."""
    g = rng(seed)
    v = g.normal(size=(lattice, lattice, lattice, 3))
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    P = v[..., :, None] * v[..., None, :]           # (L, L, L, 3, 3), index [z, y, x]
    iz, fz = _lattice_coords(n, lattice)
    eps = 1.0 / kappa ** 2
    res = np.empty((6, n, n, n), dtype=dtype)
    for z in range(n):
        out = np.zeros((n, n, 3, 3))
        for dz in (0, 1):
            wz = fz[z] if dz else 1 - fz[z]
            for dy in (0, 1):
                wy = (fz if dy else 1 - fz)[:, None, None, None]
                for dx in (0, 1):
                    wx = (fz if dx else 1 - fz)[None, :, None, None]
                    blk = P[iz[z] + dz][iz + dy][:, iz + dx]
                    out += wz * wy * wx * blk
        D = eps * np.eye(3) + (1 - eps) * out
        for k, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
            res[k, z] = D[..., a, b]
    return res


def smooth_field2d(ny, nx, seed, kappa_min=1.0, kappa_max=50.0, lattice=16):
    """2D SPD field with smooth random orientation and anisotropy: angles on a
    lattice^2 grid interpolated bilinearly in doubled-angle space
    (cos 2 theta, sin 2 theta), and log kappa ~ U[log kappa_min, log
    kappa_max] on the same lattice, interpolated bilinearly."""
    g = rng(seed)
    th = g.uniform(0, np.pi, (lattice, lattice))
    lk = g.uniform(np.log(kappa_min), np.log(kappa_max), (lattice, lattice))
    c2, s2 = np.cos(2 * th), np.sin(2 * th)
    iy, fy = _lattice_coords(ny, lattice)
    ix, fx = _lattice_coords(nx, lattice)

    def interp(a):
        a00 = a[iy][:, ix]
        a01 = a[iy][:, ix + 1]
        a10 = a[iy + 1][:, ix]
        a11 = a[iy + 1][:, ix + 1]
        wy = fy[:, None]
        wx = fx[None, :]
        return (1 - wy) * ((1 - wx) * a00 + wx * a01) + wy * ((1 - wx) * a10 + wx * a11)

    theta = 0.5 * np.arctan2(interp(s2), interp(c2))
    kappa = np.exp(interp(lk))
    return D_from_angle(theta, kappa)


def smooth_field2d_torch(ny, nx, seed, kappa_min=1.0, kappa_max=50.0, lattice=16, device="cuda",
                        dtype=None):
    """smooth_field2d evaluated with torch on `device` (FP64 arithmetic, the
    same lattice draws); for large benchmark inputs.  Returns a tensor
    (3, ny, nx) of `dtype` (default float32)."""
    import torch
    g = rng(seed)
    th = g.uniform(0, np.pi, (lattice, lattice))
    lk = g.uniform(np.log(kappa_min), np.log(kappa_max), (lattice, lattice))
    iy, fy = _lattice_coords(ny, lattice)
    ix, fx = _lattice_coords(nx, lattice)
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device)
    iy, ix, fy, fx = (torch.as_tensor(iy, device=device), torch.as_tensor(ix, device=device),
                      T(fy)[:, None], T(fx)[None, :])

    def interp(a):
        a = T(a)
        a00 = a[iy][:, ix]
        a01 = a[iy][:, ix + 1]
        a10 = a[iy + 1][:, ix]
        a11 = a[iy + 1][:, ix + 1]
        return (1 - fy) * ((1 - fx) * a00 + fx * a01) + fy * ((1 - fx) * a10 + fx * a11)

    theta = 0.5 * torch.atan2(interp(np.sin(2 * th)), interp(np.cos(2 * th)))
    lam2 = 1.0 / torch.exp(interp(lk)) ** 2
    c, s_ = torch.cos(theta), torch.sin(theta)
    D = torch.stack([c * c + lam2 * s_ * s_, (1.0 - lam2) * c * s_, s_ * s_ + lam2 * c * c])
    return D.to(dtype or torch.float32)


def restoration_problem(N, kappa, alpha=1.0 / 3.0):
    """The restoration test with a known solution (Sec. 5, "A test case with an
    explicit solution") on the N x N cell-centred grid of [0,1)^2: the
    tensor field D = [[1, s], [s, s^2 + kappa^-2]], s = 2 pi alpha sin(2 pi x),
    and the transported stripe image v(x, y) = 1 if y + alpha cos(2 pi x) < 1/2.
    Returns (D planes (3, N, N), v (N, N), the stripe coordinate
    y + alpha cos(2 pi x) (N, N)); arrays indexed [y, x]."""
    c = (np.arange(N) + 0.5) / N
    X, Y = np.meshgrid(c, c)
    s = 2 * np.pi * alpha * np.sin(2 * np.pi * X)
    D = np.stack([np.ones_like(s), s, s * s + kappa ** -2.0])
    Yf = Y + alpha * np.cos(2 * np.pi * X)
    return D, (Yf < 0.5).astype(np.float64), Yf


def radial3d(n, seed, R=0.5, noise_var=0.5):
    """The synthetic 3D image of the paper's 3D experiments on the n^3
    cell-centred grid of [0,1]^3: u0 = cos(2 (r/R)^3) with r = |x|, and
    u0 + Gaussian noise of variance noise_var.  Returns (u0, noisy), [z, y, x]."""
    c = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    u0 = np.cos(2.0 * (r / R) ** 3)
    return u0, u0 + rng(seed).normal(0.0, np.sqrt(noise_var), u0.shape)


def shells3d(shape, seed, noise=0.15, n_blobs=6):
    """Stand-in for the paper's 256 x 256 x 100 MRI volume (Sec. 5, 3D MRI
    data), which is not available here: nested ellipsoidal shells with
    piecewise-constant intensities (outer layer 0.6, shell 1.0, interior
    0.4) and n_blobs inner balls of random centre, radius and intensity,
    on the cell-centred grid of shape (nz, ny, nx) over a unit box per axis;
    plus N(0, noise^2) per voxel.  Returns (clean, noisy), [z, y, x]."""
    g = rng(seed)
    axes = [(np.arange(n) + 0.5) / n - 0.5 for n in shape]
    Z, Y, X = np.meshgrid(*axes, indexing="ij")
    r = np.sqrt((X / 0.42) ** 2 + (Y / 0.46) ** 2 + (Z / 0.45) ** 2)
    u = np.zeros(shape)
    u[r < 1.0] = 0.6
    u[r < 0.93] = 1.0
    u[r < 0.85] = 0.4
    for _ in range(n_blobs):
        c = g.uniform(-0.25, 0.25, 3)
        rad = g.uniform(0.04, 0.1)
        val = g.uniform(0.1, 0.9)
        u[np.sqrt((Z - c[0]) ** 2 + (Y - c[1]) ** 2 + (X - c[2]) ** 2) < rad] = val
    return u, u + g.normal(0.0, noise, shape)


def batch_items(seed=100, n_images=64, n_volumes=8, img_sides=(256, 2048), vol_sides=(64, 192),
                kappa=(5.0, 100.0)):
    """Uneven batch: per item a dict with its shape, tensor-field seed and
    anisotropy; images of side ~ U{256..2048}, volumes ~ U{64..192}."""
    g = rng(seed)
    items = []
    for i in range(n_images):
        s = int(g.integers(img_sides[0], img_sides[1] + 1))
        items.append({"dim": 2, "shape": (s, s), "seed": seed + i,
                      "kappa": float(g.uniform(*kappa))})
    for i in range(n_volumes):
        s = int(g.integers(vol_sides[0], vol_sides[1] + 1))
        items.append({"dim": 3, "shape": (s, s, s), "seed": seed + n_images + i,
                      "kappa": float(g.uniform(*kappa))})
    return items


def random_spd2(n, seed, kappa_max=100.0):
    """n random 2D tensors with uniform orientation and kappa in [1, kappa_max]
    (log-uniform), scaled by a random positive factor."""
    g = rng(seed)
    th = g.uniform(0, np.pi, n)
    k = np.exp(g.uniform(0, np.log(kappa_max), n))
    s = np.exp(g.uniform(-3, 3, n))
    return D_from_angle(th, k) * s


def random_spd3(n, seed, kappa_max=20.0):
    """n random 3D tensors R diag(1, k1^-2, k2^-2) R^T with R uniform (QR of a
    Gaussian matrix) and k1, k2 log-uniform in [1, kappa_max]."""
    g = rng(seed)
    out = np.zeros((6, n))
    for i in range(n):
        Q, R = np.linalg.qr(g.normal(size=(3, 3)))
        Q = Q * np.sign(np.diag(R))
        lam = np.array([1.0, np.exp(-2 * g.uniform(0, np.log(kappa_max))),
                        np.exp(-2 * g.uniform(0, np.log(kappa_max)))])
        D = (Q * lam) @ Q.T
        out[:, i] = [D[0, 0], D[1, 1], D[2, 2], D[0, 1], D[0, 2], D[1, 2]]
    return out
