"""Seeded synthetic inputs shaped like the paper's volumes (no method arithmetic here).

The paper's inputs are DNS volumes of a premixed hydrogen/ammonia/nitrogen flame and of
channel flow (Sec. 6); none of them is available, so these generators stand in for them.
Both the oracle tests and the CUDA path consume the same generated arrays; nothing here
implements any step of the tessellation.

Volumes are float32 arrays of shape (nz, ny, nx), x fastest.  Generators run with torch
on the device they are given (CPU or CUDA) so large volumes are built quickly on the GPU.

Recipes (the five workloads):
  blobs   : sum of Gaussian blobs, centres U[0, side)^3, sigma U(3, 10), amplitude
            U(0.5, 1), plus N(0, 0.02) noise.  24 blobs per 64^3 of volume.
  flame   : u = isotropic spectral field with amplitude ~ |k|^(-11/6) (E(k) ~ k^(-5/3))
            and a dissipation-range cutoff exp(-2.6 k eta), eta = 2 voxels, random phases,
            unit std; f = (1 + tanh((x - nx/2 + 24 u) / 8)) / 2, a progress-variable-like
            front about 16 voxels thick.  Recipe "sharp": eta = 0 (no cutoff) and tanh
            width 4, which shatters the thin isobands into very many components.
  corr    : m correlated Gaussian variables x = mu + L z, L L^T = A A^T / m + 0.1 I.
"""
import math

import numpy as np
import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def blob_field(dims, seed, device="cpu", n_blobs=None, noise=0.02, window=True):
    """Sum of Gaussian blobs plus Gaussian noise.  dims = (nx, ny, nz)."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    vol = nx * ny * nz
    if n_blobs is None:
        n_blobs = max(4, int(round(24.0 * vol / 64 ** 3)))
    cen = rng.uniform(0.0, 1.0, size=(n_blobs, 3)) * np.array([nx, ny, nz])
    sig = rng.uniform(3.0, 10.0, size=n_blobs)
    amp = rng.uniform(0.5, 1.0, size=n_blobs)
    f = torch.zeros((nz, ny, nx), dtype=torch.float32, device=device)
    xs = torch.arange(nx, dtype=torch.float32, device=device)
    ys = torch.arange(ny, dtype=torch.float32, device=device)
    zs = torch.arange(nz, dtype=torch.float32, device=device)
    for b in range(n_blobs):
        cx, cy, cz = cen[b]
        s = float(sig[b])
        if window:
            r = 4.0 * s
            x0, x1 = max(0, int(math.floor(cx - r))), min(nx, int(math.ceil(cx + r)) + 1)
            y0, y1 = max(0, int(math.floor(cy - r))), min(ny, int(math.ceil(cy + r)) + 1)
            z0, z1 = max(0, int(math.floor(cz - r))), min(nz, int(math.ceil(cz + r)) + 1)
        else:
            x0, x1, y0, y1, z0, z1 = 0, nx, 0, ny, 0, nz
        if x0 >= x1 or y0 >= y1 or z0 >= z1:
            continue
        gx = torch.exp(-((xs[x0:x1] - cx) ** 2) / (2 * s * s))
        gy = torch.exp(-((ys[y0:y1] - cy) ** 2) / (2 * s * s))
        gz = torch.exp(-((zs[z0:z1] - cz) ** 2) / (2 * s * s))
        f[z0:z1, y0:y1, x0:x1] += float(amp[b]) * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    if noise > 0:
        f += noise * torch.randn((nz, ny, nx), generator=_gen(seed + 7919, device), device=device)
    return f


def spectral_field(dims, seed, device="cpu", slope=-11.0 / 6.0, eta=2.0):
    """Isotropic Gaussian random field, unit std, spectral amplitude |k|^slope (inertial
    range) times exp(-2.6 k eta) (the dissipation range of Pope's model spectrum,
    exp(-5.2 k eta) in energy, with Kolmogorov scale eta in voxels), so that the field is
    smooth at the grid scale like a resolved DNS.  eta = 0 disables the cutoff."""
    nx, ny, nz = dims
    g = _gen(seed, device)
    kz = torch.fft.fftfreq(nz, device=device).view(nz, 1, 1)
    ky = torch.fft.fftfreq(ny, device=device).view(1, ny, 1)
    kx = torch.fft.rfftfreq(nx, device=device).view(1, 1, nx // 2 + 1)
    k = torch.sqrt((kx * nx) ** 2 + (ky * ny) ** 2 + (kz * nz) ** 2)
    kphys = 2.0 * math.pi * torch.sqrt(kx ** 2 + ky ** 2 + kz ** 2)  # radians per voxel
    k[0, 0, 0] = 1.0
    amp = k.pow(slope)
    if eta > 0:
        amp = amp * torch.exp(-2.6 * kphys * eta)
    del kphys
    amp[0, 0, 0] = 0.0
    del k
    re = torch.randn(amp.shape, generator=g, device=device)
    im = torch.randn(amp.shape, generator=g, device=device)
    spec = torch.complex(re * amp, im * amp)
    del re, im, amp
    u = torch.fft.irfftn(spec, s=(nz, ny, nx))
    del spec
    u = u - u.mean()
    u = u / u.std()
    return u.to(torch.float32).contiguous()


FLAME_RECIPES = {
    # a resolved front: dissipation-range cutoff (eta = 2 voxels), tanh width 8
    "resolved": dict(eta=2.0, width=8.0),
    # a sharp front: pure k^-5/3 amplitudes to the grid scale, tanh width 4;
    # it breaks the thin isobands into very many small components
    "sharp": dict(eta=0.0, width=4.0),
}


def flame_field(dims, seed, device="cpu", width=8.0, eta=2.0):
    """Progress-variable-like flame front wrinkled by spectral turbulence.  Returns (f, u).
    The tanh width (8 voxels) makes the front about 16 voxels thick, resolved like a DNS flame."""
    nx, ny, nz = dims
    u = spectral_field(dims, seed, device, eta=eta)
    x = torch.arange(nx, dtype=torch.float32, device=device).view(1, 1, nx)
    f = 0.5 * (1.0 + torch.tanh((x - nx / 2.0 + 24.0 * u) / width))
    return f.to(torch.float32).contiguous(), u


def correlated_aux(dims, m, seed, device="cpu", chunk=1 << 24):
    """m correlated Gaussian variables, shape (m, nz, ny, nx): x = mu + L z."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, m))
    cov = A @ A.T / m + 0.1 * np.eye(m)
    L = np.linalg.cholesky(cov)
    mu = rng.uniform(-2.0, 2.0, size=m)
    Lt = torch.tensor(L, dtype=torch.float32, device=device)
    mut = torch.tensor(mu, dtype=torch.float32, device=device).view(m, 1)
    n = nx * ny * nz
    out = torch.empty((m, n), dtype=torch.float32, device=device)
    g = _gen(seed + 1, device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        z = torch.randn((m, e - s), generator=g, device=device)
        out[:, s:e] = Lt @ z + mut
    return out.view(m, nz, ny, nx), cov, mu


# --------------------------------------------------------------------------- workloads
def blobs_workload(side=64, seed=1, device="cpu", n_aux=3):
    """64^3 sum of 24 Gaussian blobs + N(0, 0.02) noise; 4 isovalues -> 5 bands; 512 voxels
    per site, uniform weight; 10 Lloyd iterations; aux = (f, second blob field, N(0,1))."""
    dims = (side, side, side) if np.isscalar(side) else tuple(side)
    f = blob_field(dims, seed, device)
    aux = [f]
    if n_aux > 1:
        aux.append(blob_field(dims, seed + 100, device))
    if n_aux > 2:
        aux.append(torch.randn(f.shape, generator=_gen(seed + 200, device), device=device))
    return dict(name="blobs%dx%dx%d" % dims, dims=dims, field=f,
                iso=np.array([0.2, 0.4, 0.6, 0.8], np.float32), gamma=0, voxels_per_site=512,
                strat_block=16, rng_seed=seed, n_iters=10, n_bins=32,
                aux=torch.stack(aux[:n_aux]) if n_aux else torch.zeros((0,) + f.shape, device=device))


def flame_workload(side=512, seed=2, device="cpu", n_aux=16, n_iters=30, recipe="resolved"):
    """512^3 spectral-turbulence flame; 8 isovalues i/9; weight |grad f| (gamma 1);
    4096 voxels per site; 30 Lloyd iterations; 16 aux = (f, u, 14 spectral fields).
    recipe: "resolved" (default) or "sharp" (see FLAME_RECIPES)."""
    dims = (side, side, side) if np.isscalar(side) else tuple(side)
    f, u = flame_field(dims, seed, device, **FLAME_RECIPES[recipe])
    aux = torch.empty((n_aux,) + f.shape, dtype=torch.float32, device=device)
    if n_aux > 0:
        aux[0] = f
    if n_aux > 1:
        aux[1] = u
    del u
    for j in range(2, n_aux):
        aux[j] = spectral_field(dims, seed * 1000 + j, device)
    return dict(name="flame%dx%dx%d%s" % (dims + ("" if recipe == "resolved" else "-" + recipe,)), dims=dims, field=f,
                iso=(np.arange(1, 9, dtype=np.float32) / np.float32(9.0)).astype(np.float32), gamma=1,
                voxels_per_site=4096, strat_block=16, rng_seed=seed, n_iters=n_iters, n_bins=32, aux=aux)


def block_batch(n_blocks=64, seed=3, lo=32, hi=256, device="cpu"):
    """Independent blocks with sides drawn per axis from U{lo..hi}, blob fields (blob count
    24 V / 64^3, at least 4), k ~ U{2..12} isovalues i/(k+1), 512 voxels per site."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_blocks):
        dims = tuple(int(v) for v in rng.integers(lo, hi + 1, size=3))
        k = int(rng.integers(2, 13))
        f = blob_field(dims, seed * 100000 + b, device)
        aux = torch.stack([f, blob_field(dims, seed * 100000 + b + 50000, device),
                           torch.randn(f.shape, generator=_gen(seed * 7 + b, device), device=device)])
        out.append(dict(dims=dims, field=f, iso=(np.arange(1, k + 1) / (k + 1)).astype(np.float32), gamma=0,
                        voxels_per_site=512, strat_block=16, rng_seed=seed * 1000 + b, n_iters=20, n_bins=32,
                        aux=aux))
    return out


class CropPool:
    """Resident master volumes a request stream is cut from: one blob field and `n_aux` blob
    variables of side `side` (the served requests are blocks of one large simulation, each a
    sub-volume at a seeded offset).  `request_data(req)` copies a request's field and variables
    out of the masters on the current stream (a few device copies, no host work), so a server
    can build a request's inputs when it admits it."""

    def __init__(self, side=512, n_aux=16, seed=7, device="cpu"):
        self.side = side
        self.field = blob_field((side, side, side), seed, device)
        self.aux = [blob_field((side, side, side), seed + 1 + j, device, n_blobs=8, noise=0.1) for j in range(n_aux)]

    def request_data(self, req):
        nx, ny, nz = req["dims"]
        rng = np.random.default_rng(req["seed"])
        x0, y0, z0 = (int(rng.integers(0, self.side - n + 1)) for n in (nx, ny, nz))
        cut = lambda v: v[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx].contiguous()
        return cut(self.field), [cut(self.aux[j]) for j in range(req["n_aux"])]


def request_stream(n_requests=1000, rate=50.0, seed=5, lo=64, hi=512):
    """Poisson arrivals (exponential gaps, mean rate per second) of decomposition requests.
    Returns descriptors only (fields are generated by the caller with blob_field)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    reqs = []
    for i in range(n_requests):
        dims = tuple(int(v) for v in rng.integers(lo, hi + 1, size=3))
        k = int(rng.integers(2, 11))
        reqs.append(dict(arrival=float(t[i]), dims=dims, seed=seed * 100000 + i,
                         iso=(np.arange(1, k + 1) / (k + 1)).astype(np.float32), n_aux=int(rng.integers(0, 17)),
                         n_iters=int(rng.integers(10, 31)), voxels_per_site=512, strat_block=16, gamma=0,
                         n_bins=32))
    return reqs
