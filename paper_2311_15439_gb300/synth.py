"""Seeded synthetic inputs for the encoding workloads.

This module holds none of the encoding's arithmetic: it only draws points,
table values, upstream gradients and procedural targets from numpy's PCG64
generator, so that the CUDA path and the FP64 oracle can be fed the same bits.
All arrays are host numpy arrays; callers move them to the device.

Workload recipes (shapes and distributions of the paper's tasks, Sec. 6):

* ``uniform_points``   -- P points uniform in [0, 1)^d, binary32.
* ``edge_points``      -- points on the faces x = 0 and x = 1, on lattice
  planes and with tied coordinates (the degenerate cases of the subdivision).
* ``sdf_points``       -- half uniform in [0,1)^3, half within 0.01 of the
  surface of a seeded union of spheres and tori (SDF-style sampling).
* ``uniform_tables``   -- [L, T, F] values U(-a, a) stored as fp32 / fp16 /
  bf16 (bf16 is returned as the binary32 values it represents plus its raw
  uint16 bits).
* ``normal_grads``     -- upstream gradients N(0, 1).
* ``camera_rays``      -- rays from a sphere of radius 1.2 around the unit cube's centre
  towards random targets inside the cube, with the entry and exit distances of the
  cube [0,1]^3 (the volumetric workload of Sec. 6.2).
* ``BlobScene``        -- a volumetric scene: density a seeded sum of Gaussian blobs inside
  the unit cube, colour a smooth function of position (the training target of Sec. 6.2's
  setting: ray colours rendered from it).
* ``ProceduralImage``  -- an RGB image defined analytically as a seeded sum of
  sinusoids plus bilinear value noise on a coarse lattice; it stands in for the
  gigapixel photograph of Sec. 6.1, which is not available here.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_points(P: int, d: int, seed: int) -> np.ndarray:
    return rng(seed).random((P, d), dtype=np.float32)


def edge_points(d: int, seed: int, per_kind: int = 64) -> np.ndarray:
    """Degenerate inputs: corners/faces of the unit cube, ties, tiny and near-1 values."""
    g = rng(seed)
    pts = []
    # faces x_i = 0 and x_i = 1
    for i in range(d):
        for val in (0.0, 1.0):
            p = g.random((per_kind, d), dtype=np.float32)
            p[:, i] = val
            pts.append(p)
    # corners
    for bits in range(1 << d):
        pts.append(np.array([[(bits >> i) & 1 for i in range(d)]], dtype=np.float32))
    # all coordinates tied
    t = g.random((per_kind, 1), dtype=np.float32)
    pts.append(np.repeat(t, d, axis=1))
    # pairs tied
    p = g.random((per_kind, d), dtype=np.float32)
    p[:, 1] = p[:, 0]
    pts.append(p)
    # coordinates on coarse dyadic values (land exactly on lattice planes at many levels)
    k = g.integers(0, 65, size=(per_kind, d))
    pts.append((k / 64.0).astype(np.float32))
    # values just below 1 and just above 0
    pts.append(np.full((1, d), np.nextafter(np.float32(1), np.float32(0)), dtype=np.float32))
    pts.append(np.full((1, d), np.float32(1e-30), dtype=np.float32))
    return np.concatenate(pts, axis=0)


def fp32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round binary32 to bfloat16 (nearest, ties to even); returns the uint16 bits."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    rounding = ((u >> 16) & 1) + np.uint32(0x7FFF)
    return ((u + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_fp32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def uniform_tables(L: int, T: int, F: int, seed: int, dtype: str = "f32", scale: float = 1e-4):
    """Returns (values, storage): values as binary32 exactly equal to what is stored,
    storage as the array to copy to the device (float32, float16 or uint16 bf16 bits)."""
    v = rng(seed).uniform(-scale, scale, size=(L, T, F)).astype(np.float32)
    if dtype == "f32":
        return v, v
    if dtype == "f16":
        h = v.astype(np.float16)
        return h.astype(np.float32), h
    if dtype == "bf16":
        bits = fp32_to_bf16_bits(v)
        return bf16_bits_to_fp32(bits), bits
    raise ValueError(dtype)


def normal_grads(P: int, n: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal((P, n), dtype=np.float32)


class SphereTorusScene:
    """Seeded union of spheres and tori (the SDF-style workload's surface): centres in
    [0.2, 0.8]^3, radii 0.03..0.15, tori in the xy plane with minor radius r/3.
    ``sdf(x)`` is the signed distance of the union (minimum over shapes), float32 [P, 1]."""

    def __init__(self, seed: int, n_shapes: int = 32):
        g = rng(seed)
        self.kinds = g.integers(0, 2, size=n_shapes)
        self.centres = g.uniform(0.2, 0.8, size=(n_shapes, 3))
        self.radii = g.uniform(0.03, 0.15, size=n_shapes)

    def sdf(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        best = np.full(x.shape[0], np.inf)
        for kind, c, r in zip(self.kinds, self.centres, self.radii):
            p = x - c
            if kind == 0:
                dist = np.linalg.norm(p, axis=1) - r
            else:
                q = np.stack([np.hypot(p[:, 0], p[:, 1]) - r, p[:, 2]], axis=1)
                dist = np.linalg.norm(q, axis=1) - r / 3.0
            best = np.minimum(best, dist)
        return best.astype(np.float32)[:, None]

    def sdf_torch(self, x):
        """``sdf`` evaluated with torch on x's device in binary32 (float32 tensor [P, 3] -> [P, 1])."""
        import torch
        best = torch.full((x.shape[0],), float("inf"), dtype=torch.float32, device=x.device)
        for kind, c, r in zip(self.kinds, self.centres, self.radii):
            p = x - torch.as_tensor(c, dtype=torch.float32, device=x.device)
            if kind == 0:
                dist = torch.linalg.norm(p, dim=1) - float(r)
            else:
                q = torch.stack([torch.hypot(p[:, 0], p[:, 1]) - float(r), p[:, 2]], dim=1)
                dist = torch.linalg.norm(q, dim=1) - float(r) / 3.0
            best = torch.minimum(best, dist)
        return best[:, None]

    def sample_torch(self, P: int, gen, band: float = 0.01):
        """P training points on ``gen``'s device: half uniform in [0,1)^3, half within ``band`` of
        this scene's surface (a random shape, a random point on it, a random normal offset), the
        recipe of ``sdf_points`` applied to this scene; float32 [P, 3]."""
        import torch
        dev = gen.device
        n_uni = P // 2
        n_sur = P - n_uni
        uni = torch.rand((n_uni, 3), generator=gen, device=dev)
        which = torch.randint(0, len(self.kinds), (n_sur,), generator=gen, device=dev)
        kinds = torch.as_tensor(self.kinds, device=dev)[which]
        c = torch.as_tensor(self.centres, dtype=torch.float32, device=dev)[which]
        r = torch.as_tensor(self.radii, dtype=torch.float32, device=dev)[which]
        off = (torch.rand((n_sur,), generator=gen, device=dev) * 2 - 1) * band
        u = torch.randn((n_sur, 3), generator=gen, device=dev)
        u = u / torch.linalg.norm(u, dim=1, keepdim=True)
        angle = torch.rand((n_sur,), generator=gen, device=dev) * (2 * np.pi)
        tube = torch.rand((n_sur,), generator=gen, device=dev) * (2 * np.pi)
        sph = c + (r + off)[:, None] * u
        rm = r / 3.0 + off
        tor = torch.stack([c[:, 0] + (r + rm * torch.cos(tube)) * torch.cos(angle),
                           c[:, 1] + (r + rm * torch.cos(tube)) * torch.sin(angle),
                           c[:, 2] + rm * torch.sin(tube)], dim=1)
        sur = torch.where((kinds == 0)[:, None], sph, tor).clamp_(0.0, float(np.nextafter(np.float32(1), 0)))
        pts = torch.cat([uni, sur])
        return pts[torch.randperm(P, generator=gen, device=dev)]

    def sample(self, P: int, seed: int, band: float = 0.01) -> np.ndarray:
        """Host (numpy) form of ``sample_torch``'s recipe: half uniform in [0,1)^3, half within
        ``band`` of this scene's surface; float32 [P, 3]."""
        g = rng(seed)
        n_uni = P // 2
        n_sur = P - n_uni
        uni = g.random((n_uni, 3))
        which = g.integers(0, len(self.kinds), size=n_sur)
        c, r = self.centres[which], self.radii[which]
        off = g.uniform(-band, band, size=n_sur)
        u = g.standard_normal((n_sur, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        angle = g.uniform(0.0, 2 * np.pi, size=n_sur)
        tube = g.uniform(0.0, 2 * np.pi, size=n_sur)
        sph = c + (r + off)[:, None] * u
        rm = r / 3.0 + off
        tor = np.stack([c[:, 0] + (r + rm * np.cos(tube)) * np.cos(angle),
                        c[:, 1] + (r + rm * np.cos(tube)) * np.sin(angle),
                        c[:, 2] + rm * np.sin(tube)], axis=1)
        sur = np.clip(np.where((self.kinds[which] == 0)[:, None], sph, tor), 0.0, np.nextafter(1.0, 0.0))
        return np.concatenate([uni, sur]).astype(np.float32)


def sdf_points(P: int, seed: int, n_shapes: int = 32, band: float = 0.01) -> np.ndarray:
    """Half uniform in [0,1)^3, half within ``band`` of a seeded union of spheres and tori."""
    g = rng(seed)
    n_uni = P // 2
    n_sur = P - n_uni
    pts = [g.random((n_uni, 3))]
    kinds = g.integers(0, 2, size=n_shapes)
    centres = g.uniform(0.2, 0.8, size=(n_shapes, 3))
    radii = g.uniform(0.03, 0.15, size=n_shapes)
    which = g.integers(0, n_shapes, size=n_sur)
    u = g.standard_normal((n_sur, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    off = g.uniform(-band, band, size=(n_sur, 1))
    angle = g.uniform(0.0, 2 * np.pi, size=n_sur)
    tube = g.uniform(0.0, 2 * np.pi, size=n_sur)
    sur = np.empty((n_sur, 3))
    sph = kinds[which] == 0
    r = radii[which][:, None]
    sur[sph] = centres[which][sph] + (r[sph] + off[sph]) * u[sph]
    # torus in the xy plane: major radius r, minor radius r/3
    tor = ~sph
    rr, rm = r[tor, 0], r[tor, 0] / 3.0 + off[tor, 0]
    sur[tor, 0] = centres[which][tor, 0] + (rr + rm * np.cos(tube[tor])) * np.cos(angle[tor])
    sur[tor, 1] = centres[which][tor, 1] + (rr + rm * np.cos(tube[tor])) * np.sin(angle[tor])
    sur[tor, 2] = centres[which][tor, 2] + rm * np.sin(tube[tor])
    pts.append(np.clip(sur, 0.0, np.nextafter(1.0, 0.0)))
    out = np.concatenate(pts).astype(np.float32)
    return out[g.permutation(P)]


def camera_rays(R: int, seed: int):
    """(origins [R,3], unit directions [R,3], t_near [R], t_far [R]) float32: origins on the
    sphere of radius 1.2 about (0.5, 0.5, 0.5), each aimed at a uniform point of [0.25, 0.75]^3;
    [t_near, t_far] is the ray's segment inside [0,1]^3 (slab test in FP64)."""
    g = rng(seed)
    u = g.standard_normal((R, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    o = 0.5 + 1.2 * u
    target = g.uniform(0.25, 0.75, size=(R, 3))
    d = target - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    with np.errstate(divide="ignore"):
        inv = 1.0 / d
    t0 = (0.0 - o) * inv
    t1 = (1.0 - o) * inv
    tn = np.maximum(np.minimum(t0, t1).max(axis=1), 0.0)
    tf = np.maximum(t0, t1).min(axis=1)
    return (o.astype(np.float32), d.astype(np.float32), tn.astype(np.float32), tf.astype(np.float32))


class BlobScene:
    """Density sigma(x) = sum_k a_k exp(-|x - m_k|^2 / (2 s_k^2)) over seeded blobs (centres in
    [0.3, 0.7]^3, widths 0.03..0.1, peaks 20..80) and colour c(x) = 0.5 + 0.5 sin(omega x + phi)
    per channel; ``field(x)`` returns (sigma [P], rgb [P, 3]) in FP64."""

    def __init__(self, seed: int, n_blobs: int = 12):
        g = rng(seed)
        self.m = g.uniform(0.3, 0.7, size=(n_blobs, 3))
        self.s = g.uniform(0.03, 0.1, size=n_blobs)
        self.a = g.uniform(20.0, 80.0, size=n_blobs)
        self.omega = g.uniform(2.0, 8.0, size=(3, 3))
        self.phi = g.uniform(0.0, 2 * np.pi, size=3)

    def field(self, x: np.ndarray):
        x = np.asarray(x, dtype=np.float64)
        d2 = ((x[:, None, :] - self.m[None, :, :]) ** 2).sum(axis=2)
        sigma = (self.a[None, :] * np.exp(-d2 / (2.0 * self.s[None, :] ** 2))).sum(axis=1)
        rgb = 0.5 + 0.5 * np.sin(x @ self.omega.T + self.phi[None, :])
        return sigma, rgb


class ProceduralImage:
    """RGB image of ``size`` x ``size`` pixels defined analytically (no pixel array):
    a seeded sum of ``n_waves`` sinusoids per channel plus bilinear value noise on
    a 64 x 64 lattice, mapped to [0, 1].  ``sample(x)`` evaluates it at points
    x in [0,1)^2 (pixel-centre snapped), returning float32 [P, 3]."""

    def __init__(self, seed: int, size: int = 16384, n_waves: int = 64):
        g = rng(seed)
        self.size = size
        self.freq = g.uniform(1.0, 400.0, size=(3, n_waves, 1)) * g.choice([-1, 1], size=(3, n_waves, 2))
        self.dirs = g.standard_normal((3, n_waves, 2))
        self.dirs /= np.linalg.norm(self.dirs, axis=2, keepdims=True)
        self.phase = g.uniform(0, 2 * np.pi, size=(3, n_waves))
        self.amp = g.uniform(0.2, 1.0, size=(3, n_waves)) / n_waves
        self.noise = g.random((3, 65, 65))

    def sample(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        px = (np.floor(x * self.size) + 0.5) / self.size
        out = np.empty((x.shape[0], 3))
        gx = px[:, 0] * 64.0
        gy = px[:, 1] * 64.0
        ix = np.minimum(gx.astype(np.int64), 63)
        iy = np.minimum(gy.astype(np.int64), 63)
        fx, fy = gx - ix, gy - iy
        for ch in range(3):
            k = self.dirs[ch] * np.abs(self.freq[ch])                # [W, 2]
            arg = px @ k.T + self.phase[ch]                          # [P, W]
            s = np.sin(arg) @ self.amp[ch]
            nz = self.noise[ch]
            vn = ((1 - fx) * (1 - fy) * nz[ix, iy] + fx * (1 - fy) * nz[ix + 1, iy]
                  + (1 - fx) * fy * nz[ix, iy + 1] + fx * fy * nz[ix + 1, iy + 1])
            out[:, ch] = 0.5 + 0.35 * s + 0.3 * (vn - 0.5)
        return np.clip(out, 0.0, 1.0).astype(np.float32)

    def sample_torch(self, x):
        """``sample`` evaluated with torch on x's device in binary32 (for generating many training
        batches on the GPU; within about 1e-5 of the FP64 ``sample``).  x: float32 tensor [P, 2]."""
        import torch
        dev = x.device
        px = (torch.floor(x * self.size) + 0.5) / self.size
        gx, gy = px[:, 0] * 64.0, px[:, 1] * 64.0
        ix = torch.clamp(gx.to(torch.int64), max=63)
        iy = torch.clamp(gy.to(torch.int64), max=63)
        fx, fy = gx - ix.to(gx.dtype), gy - iy.to(gy.dtype)
        out = torch.empty((x.shape[0], 3), dtype=torch.float32, device=dev)
        for ch in range(3):
            k = torch.as_tensor(self.dirs[ch] * np.abs(self.freq[ch]), dtype=torch.float32, device=dev)
            ph = torch.as_tensor(self.phase[ch], dtype=torch.float32, device=dev)
            amp = torch.as_tensor(self.amp[ch], dtype=torch.float32, device=dev)
            s = torch.sin(px @ k.T + ph) @ amp
            nz = torch.as_tensor(self.noise[ch], dtype=torch.float32, device=dev)
            vn = ((1 - fx) * (1 - fy) * nz[ix, iy] + fx * (1 - fy) * nz[ix + 1, iy]
                  + (1 - fx) * fy * nz[ix, iy + 1] + fx * fy * nz[ix + 1, iy + 1])
            out[:, ch] = 0.5 + 0.35 * s + 0.3 * (vn - 0.5)
        return out.clamp_(0.0, 1.0)
