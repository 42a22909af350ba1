"""Seeded synthetic inputs for the holographic Gaussian renderer.

This module is shared by the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2506_08350_b300``).  It holds only input generation: scenes, cameras,
optics and upstream gradients.  None of the method's arithmetic (projection,
compositing, propagation, gradients) lives here.

Scene recipe (stands in for the paper's datasets, which are not available):

* camera 0 at the origin, OpenCV axes (x right, y down, z forward),
  f_x = f_y = (W/2)/tan(30 deg) (60 deg horizontal field of view),
  c_x = (W-1)/2, c_y = (H-1)/2;
* means uniform in the camera-0 frustum volume between 1 and 3 m:
  z = (1 + 26 u)^(1/3), pixel position uniform over the image, back-projected;
* log-scales N(-4, 0.5) iid per axis;
* rotations: normalised N(0,1)^4 quaternions (w, x, y, z);
* amplitude U[0,1] per wavelength, phase U[0, 2 pi) per wavelength;
* opacity U[0.1, 1) stored as a logit;
* plane logits -((z - zbar_l)/Delta)^2 with zbar_l the centres of L equal depth
  bins over [1, 3] m, so the argmax is the depth bin.

All generators use numpy's PCG64 with explicit seeds.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WAVELENGTHS_RGB = (639e-9, 515e-9, 473e-9)


@dataclasses.dataclass
class Optics:
    """Hologram-plane sampling and the depth planes (paper Sec. 3, background
    paragraph on the hologram plane, and the layer-construction paragraph)."""

    H: int
    W: int
    wavelengths: tuple  # metres, one per colour channel
    plane_z: tuple  # metres, distance Z_l from plane l to the hologram plane
    pitch: float = 8e-6  # metres, square pixels
    band_limit: int = 0  # 1: Matsushima-Shimobaba band limit on top of the evanescent cut
    padding: int = 0  # 1: propagate on the 2x zero-padded grid (linear convolution)

    @property
    def C(self) -> int:
        return len(self.wavelengths)

    @property
    def L(self) -> int:
        return len(self.plane_z)


@dataclasses.dataclass
class Workload:
    name: str
    optics: Optics
    N: int
    V: int


def workload(name: str) -> Workload:
    """Named synthetic workloads (sizes of the paper-shaped scenes)."""
    if name == "c1_256_L2_N1k":
        return Workload(name, Optics(256, 256, (515e-9,), (0.0, 5e-3)), 1000, 1)
    if name == "c2_1080p_L8_N100k":
        z = tuple(float(v) for v in np.linspace(0.0, 10e-3, 8))
        return Workload(name, Optics(1080, 1920, WAVELENGTHS_RGB, z), 100_000, 1)
    if name == "c3_512_L8_N500k":
        z = tuple(float(v) for v in np.linspace(0.0, 10e-3, 8))
        return Workload(name, Optics(512, 512, WAVELENGTHS_RGB, z), 500_000, 1)
    if name == "c4_1080p_L12_N2M_V16":
        z = tuple(float(v) for v in np.linspace(0.0, 12e-3, 12))
        return Workload(name, Optics(1080, 1920, WAVELENGTHS_RGB, z), 2_000_000, 16)
    if name == "1080p_rgb_L12_N1M_V16":
        z = tuple(float(v) for v in np.linspace(0.0, 12e-3, 12))
        return Workload(name, Optics(1080, 1920, WAVELENGTHS_RGB, z), 1_000_000, 16)
    if name == "1080p_rgb_L12_N1M_V1":  # one view of the same scene (profiling captures)
        z = tuple(float(v) for v in np.linspace(0.0, 12e-3, 12))
        return Workload(name, Optics(1080, 1920, WAVELENGTHS_RGB, z), 1_000_000, 1)
    raise KeyError(name)


def intrinsics(H: int, W: int, fov_x_deg: float = 60.0) -> np.ndarray:
    f = (W / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return np.array([f, f, (W - 1) / 2.0, (H - 1) / 2.0], dtype=np.float64)


def make_gaussians(N: int, L: int, C: int, H: int, W: int, seed: int = 0,
                   fov_x_deg: float = 60.0, zmin: float = 1.0, zmax: float = 3.0,
                   log_scale_mean: float = -4.0, log_scale_std: float = 0.5) -> dict:
    """Random complex Gaussians in the camera-0 frustum; float32 SoA arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fx, fy, cx, cy = intrinsics(H, W, fov_x_deg)
    u = rng.random(N)
    a, b = zmin ** 3, zmax ** 3
    z = np.cbrt(a + (b - a) * u)
    px = rng.random(N) * W
    py = rng.random(N) * H
    means = np.stack([(px - cx) * z / fx, (py - cy) * z / fy, z], axis=1)
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(N, 3))
    q = rng.normal(size=(N, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    amplitude = rng.random((N, C))
    phase = rng.random((N, C)) * 2.0 * np.pi
    opac = 0.1 + 0.9 * rng.random(N)
    opac = np.minimum(opac, 1.0 - 1e-6)
    opacity_logits = np.log(opac / (1.0 - opac))
    edges = np.linspace(zmin, zmax, L + 1)
    centres = 0.5 * (edges[1:] + edges[:-1])
    delta = (zmax - zmin) / L
    plane_logits = -(((z[:, None] - centres[None, :]) / delta) ** 2)
    f32 = lambda x: np.ascontiguousarray(x, dtype=np.float32)
    return dict(means=f32(means), log_scales=f32(log_scales), quats=f32(q),
                opacity_logits=f32(opacity_logits), amplitude=f32(amplitude),
                phase=f32(phase), plane_logits=f32(plane_logits))


def look_at(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """World->camera 4x4 matrix, OpenCV axes (z towards the target, y down)."""
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    zc = target - eye
    zc /= np.linalg.norm(zc)
    xc = np.cross(zc, np.asarray(up, dtype=np.float64))
    if np.linalg.norm(xc) < 1e-12:
        xc = np.cross(zc, np.array([0.0, 0.0, 1.0]))
    xc /= np.linalg.norm(xc)
    yc = np.cross(zc, xc)
    Rm = np.stack([xc, yc, zc], axis=0)
    M = np.eye(4)
    M[:3, :3] = Rm
    M[:3, 3] = -Rm @ eye
    return M


def ring_cameras(K: int, radius: float = 2.0, centre=(0.0, 0.0, 2.0)) -> np.ndarray:
    """K cameras on a horizontal circle about ``centre`` looking at it; camera 0
    sits at the origin looking down +z (the identity pose)."""
    c = np.asarray(centre, dtype=np.float64)
    mats = []
    for k in range(K):
        th = 2.0 * np.pi * k / K
        eye = c + radius * np.array([np.sin(th), 0.0, -np.cos(th)])
        mats.append(look_at(eye, c))
    return np.stack(mats, axis=0)


def view_batch(V: int, H: int, W: int, seed: int = 0, jitter: float = 0.05):
    """V viewpoints near camera 0: small seeded rotations/translations of the
    identity pose, so that every view sees the scene.  View 0 is the identity."""
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    mats = [np.eye(4)]
    for _ in range(1, V):
        ang = rng.normal(scale=jitter, size=3)
        Rx = np.array([[1, 0, 0], [0, math.cos(ang[0]), -math.sin(ang[0])], [0, math.sin(ang[0]), math.cos(ang[0])]])
        Ry = np.array([[math.cos(ang[1]), 0, math.sin(ang[1])], [0, 1, 0], [-math.sin(ang[1]), 0, math.cos(ang[1])]])
        Rz = np.array([[math.cos(ang[2]), -math.sin(ang[2]), 0], [math.sin(ang[2]), math.cos(ang[2]), 0], [0, 0, 1]])
        M = np.eye(4)
        M[:3, :3] = Rz @ Ry @ Rx
        M[:3, 3] = rng.normal(scale=jitter, size=3)
        mats.append(M)
    viewmats = np.stack(mats, axis=0)
    intr = np.tile(intrinsics(H, W)[None, :], (V, 1))
    return viewmats, intr


def random_complex(shape, seed: int) -> np.ndarray:
    """CN(0,1) samples as complex64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.normal(size=shape) * math.sqrt(0.5)
    im = rng.normal(size=shape) * math.sqrt(0.5)
    return (re + 1j * im).astype(np.complex64)


def random_real(shape, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return (lo + (hi - lo) * rng.random(shape)).astype(np.float32)


def plane_masks(B: int, L: int, H: int, W: int, seed: int) -> np.ndarray:
    """Binary plane masks [B][L][H][W] float32: a smooth random depth map per
    view (a few low-frequency cosines) cut into L equal depth bins, so every
    pixel lies on exactly one plane, in connected regions as a scene's depth
    map would give."""
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.meshgrid(np.arange(H) / max(H, 1), np.arange(W) / max(W, 1), indexing="ij")
    out = np.zeros((B, L, H, W), dtype=np.float32)
    for b in range(B):
        d = np.zeros((H, W))
        for _ in range(4):
            fx, fy = rng.uniform(0.5, 3.0, size=2)
            ph = rng.uniform(0, 2 * math.pi)
            d += np.cos(2 * math.pi * (fx * xx + fy * yy) + ph)
        lo, hi = d.min(), d.max()
        lab = np.minimum((L * (d - lo) / max(hi - lo, 1e-12)).astype(int), L - 1)
        for l in range(L):
            out[b, l] = lab == l
    return out


def sample_params(gauss: dict, k: int, seed: int = 1):
    """k random (array name, flat index) pairs over the continuous parameters
    (plane logits excluded: their forward is piecewise constant)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names = ["means", "log_scales", "quats", "opacity_logits", "amplitude", "phase"]
    out = []
    for _ in range(k):
        nm = names[rng.integers(len(names))]
        out.append((nm, int(rng.integers(gauss[nm].size))))
    return out
