"""Seeded synthetic stereo sequences (input generator shared by tests and benchmark).

This module holds none of the method's arithmetic.  It ray-casts piecewise-planar
scenes -- a ground plane, a far backdrop and axis-aligned boxes, some of them
moving on their own -- from a rectified stereo rig that drives forward, and
returns left/right uint8 images, the ground-truth left disparity and the
frame-to-frame ego-motion (R, t) with X_k = R X_{k-1} + t in the left-camera
frame.  Textures are fixed to the surfaces (a texel grid in surface coordinates,
nearest sampling, a counter-based hash gives each texel a uniform value in
0..255), so both cameras see the same texture; Gaussian noise is added, then the
values are rounded and clipped.

The shapes stand in for the KITTI raw sequences used by the paper (1242 x 375,
f = 721 px, b = 0.54 m, 10 Hz), which are not available here.

Everything is torch, device-agnostic: small cases run on the CPU, the benchmark
generates its sequences on the GPU.
"""
from __future__ import annotations

import dataclasses
import math

import torch

__all__ = ["Rig", "Box", "Scene", "render", "tiny_pair", "kitti_like_sequence", "relative_motion"]


# ------------------------------------------------------------ counter-based hash

_M32 = 0xFFFFFFFF


def _mul32(x: torch.Tensor, c: int) -> torch.Tensor:
    """(x * c) mod 2^32 for 0 <= x < 2^32 without int64 overflow."""
    lo = (x & 0xFFFF) * c
    hi = (((x >> 16) * c) & 0xFFFF) << 16
    return (lo + hi) & _M32


def _mix32(x: torch.Tensor) -> torch.Tensor:
    """32-bit avalanche mix (xorshift-multiply rounds, constants from C. Wellons'
    published "lowbias32" hash)."""
    x = x & _M32
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B)
    x = x ^ (x >> 16)
    return x


def texel_value(seed: int, surface: torch.Tensor, iu: torch.Tensor, iv: torch.Tensor) -> torch.Tensor:
    """Uniform texel value in [0, 255] for integer texel coordinates."""
    h = _mix32(torch.full_like(iu, seed & _M32) ^ (surface & _M32))
    h = _mix32(h ^ (iu & _M32))
    h = _mix32(h ^ (iv & _M32))
    return (h & 0xFF).to(torch.float32)


# ------------------------------------------------------------ scene description

@dataclasses.dataclass
class Rig:
    width: int
    height: int
    f: float
    baseline: float
    cx: float | None = None
    cy: float | None = None

    def __post_init__(self):
        if self.cx is None:
            self.cx = (self.width - 1) / 2.0
        if self.cy is None:
            self.cy = (self.height - 1) / 2.0

    def K(self) -> torch.Tensor:
        return torch.tensor([[self.f, 0.0, self.cx], [0.0, self.f, self.cy], [0.0, 0.0, 1.0]],
                            dtype=torch.float32)


@dataclasses.dataclass
class Box:
    centre: tuple          # world (x, y, z) at frame 0; y grows downwards
    half: tuple            # half sizes (x, y, z)
    velocity: tuple = (0.0, 0.0, 0.0)   # world metres per frame
    texel: float = 0.05


@dataclasses.dataclass
class Scene:
    seed: int
    ground_y: float | None      # world y of the ground plane (None: no ground)
    wall_z: float               # world z of the far backdrop
    boxes: list
    ground_texel: float = 0.05
    wall_texel: float = 0.6


def _yaw(psi: float) -> torch.Tensor:
    c, s = math.cos(psi), math.sin(psi)
    return torch.tensor([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]], dtype=torch.float64)


def relative_motion(R_wc_prev, c_prev, R_wc, c):
    """(R, t) with X_k = R X_{k-1} + t for camera-to-world poses (R_wc, c)."""
    R = R_wc.T @ R_wc_prev
    t = R_wc.T @ (c_prev - c)
    return R, t


# ------------------------------------------------------------ ray casting

def render(scene: Scene, rig: Rig, R_wc: torch.Tensor, c: torch.Tensor, frame: int,
           noise_sigma: float, gen: torch.Generator | None, device="cpu"):
    """Ray-cast the left and right views; returns (left u8, right u8, left disparity f32)."""
    H, W = rig.height, rig.width
    ys, xs = torch.meshgrid(torch.arange(H, device=device, dtype=torch.float64),
                            torch.arange(W, device=device, dtype=torch.float64), indexing="ij")
    dirs_c = torch.stack([(xs - rig.cx) / rig.f, (ys - rig.cy) / rig.f, torch.ones_like(xs)], -1)
    Rw = R_wc.to(device=device, dtype=torch.float64)
    dirs = dirs_c.reshape(-1, 3) @ Rw.T          # world directions; ray depth = camera z
    cw = c.to(device=device, dtype=torch.float64)
    outs = []
    for side in (0, 1):
        origin = cw + Rw @ torch.tensor([rig.baseline * side, 0.0, 0.0], dtype=torch.float64, device=device)
        img, depth = _cast(scene, origin, dirs, frame, device)
        outs.append((img, depth))
    result = []
    for img, _ in outs:
        v = img.reshape(H, W)
        if noise_sigma > 0:
            v = v + noise_sigma * torch.randn(v.shape, generator=gen, device=device, dtype=torch.float32).to(v.dtype)
        result.append(torch.clamp(torch.round(v), 0, 255).to(torch.uint8))
    depth = outs[0][1].reshape(H, W)
    disp = (rig.f * rig.baseline / depth).to(torch.float32)
    return result[0], result[1], disp


def _cast(scene: Scene, o: torch.Tensor, dirs: torch.Tensor, frame: int, device):
    n = dirs.shape[0]
    big = torch.full((n,), float("inf"), dtype=torch.float64, device=device)
    best_t = big.clone()
    tex = torch.zeros(n, dtype=torch.float32, device=device)
    i64 = torch.int64

    def take(t, val):
        nonlocal best_t, tex
        closer = t < best_t
        best_t = torch.where(closer, t, best_t)
        tex = torch.where(closer, val, tex)

    # far backdrop: plane z = wall_z
    with torch.no_grad():
        dz = dirs[:, 2]
        t = torch.where(dz > 1e-9, (scene.wall_z - o[2]) / dz, big)
        t = torch.where(t > 0, t, big)
        p = o + t[:, None] * dirs
        iu = torch.floor(p[:, 0] / scene.wall_texel).to(i64)
        iv = torch.floor(p[:, 1] / scene.wall_texel).to(i64)
        take(t, texel_value(scene.seed, torch.full_like(iu, 1), iu, iv))
        # ground: plane y = ground_y (y down)
        if scene.ground_y is not None:
            dy = dirs[:, 1]
            t = torch.where(dy > 1e-9, (scene.ground_y - o[1]) / dy, big)
            t = torch.where(t > 0, t, big)
            p = o + t[:, None] * dirs
            iu = torch.floor(p[:, 0] / scene.ground_texel).to(i64)
            iv = torch.floor(p[:, 2] / scene.ground_texel).to(i64)
            take(t, texel_value(scene.seed, torch.full_like(iu, 2), iu, iv))
        # boxes: slab test
        inv = 1.0 / torch.where(dirs.abs() < 1e-12, torch.full_like(dirs, 1e-12), dirs)
        for bi, box in enumerate(scene.boxes):
            ctr = torch.tensor([box.centre[k] + box.velocity[k] * frame for k in range(3)],
                               dtype=torch.float64, device=device)
            half = torch.tensor(box.half, dtype=torch.float64, device=device)
            t1 = (ctr - half - o) * inv
            t2 = (ctr + half - o) * inv
            tmin = torch.minimum(t1, t2)
            tmax = torch.maximum(t1, t2)
            tnear, axis = tmin.max(dim=1)
            tfar = tmax.min(dim=1).values
            hit = (tnear < tfar) & (tnear > 0)
            t = torch.where(hit, tnear, big)
            p = o + t[:, None] * dirs - ctr            # box-local: texture moves with the box
            pu = torch.where(axis == 0, p[:, 1], p[:, 0])
            pv = torch.where(axis == 2, p[:, 1], p[:, 2])
            iu = torch.floor(pu / box.texel).to(i64)
            iv = torch.floor(pv / box.texel).to(i64)
            surf = (16 + 8 * bi + axis).to(i64)
            take(t, texel_value(scene.seed, surf, iu, iv))
    return tex, best_t


# ------------------------------------------------------------ the two workloads

def tiny_pair(seed: int = 1, device="cpu"):
    """Two frames, 384 x 128, f = 400 px, b = 0.5 m, disparities within 64.

    Frame 1 follows a 0.5 m forward camera translation; one box, about
    40 x 30 px in the image, moves on its own.  Texture noise sigma = 2.
    Returns dict(left [2,H,W] u8, right, disp [2,H,W] f32, R [2,3,3], t [2,3],
    K [3,3], baseline, rig).
    """
    g = torch.Generator().manual_seed(seed)
    rig = Rig(384, 128, 400.0, 0.5)

    def u(a, b):
        return a + (b - a) * torch.rand((), generator=g).item()

    boxes = []
    # static boxes beside the path and fronto-parallel slabs ahead
    for _ in range(5):
        side = 1 if torch.rand((), generator=g).item() < 0.5 else -1
        hx, hy, hz = u(0.4, 1.5), u(0.4, 1.2), u(0.4, 1.5)
        boxes.append(Box((side * (u(3.5, 6.0) + hx), 1.2 - hy, u(9.0, 30.0)), (hx, hy, hz), texel=u(0.03, 0.06)))
    for _ in range(2):
        boxes.append(Box((u(-2.0, 2.0), u(-1.5, 0.2), u(14.0, 35.0)), (u(0.5, 1.5), u(0.4, 1.0), 0.05),
                         texel=u(0.04, 0.08)))
    # the independently moving box: 40 x 30 px at z = 10 m is 1.0 m x 0.75 m
    mz = 10.0
    boxes.append(Box((u(-1.0, 1.0), 0.2, mz), (0.5, 0.375, 0.4), velocity=(0.3, 0.0, 0.0), texel=0.03))
    scene = Scene(seed=seed, ground_y=1.2, wall_z=60.0, boxes=boxes, ground_texel=0.04, wall_texel=0.5)
    ngen = torch.Generator(device=device).manual_seed(seed + 1000)
    Rs = [torch.eye(3, dtype=torch.float64), torch.eye(3, dtype=torch.float64)]
    cs = [torch.zeros(3, dtype=torch.float64), torch.tensor([0.0, 0.0, 0.5], dtype=torch.float64)]
    L, Rimg, D = [], [], []
    for k in range(2):
        l, r, d = render(scene, rig, Rs[k], cs[k], k, 2.0, ngen, device)
        L.append(l); Rimg.append(r); D.append(d)
    Rm = torch.stack([torch.eye(3), torch.eye(3)]).to(torch.float32)
    tv = torch.zeros(2, 3, dtype=torch.float32)
    R1, t1 = relative_motion(Rs[0], cs[0], Rs[1], cs[1])
    Rm[1] = R1.to(torch.float32)
    tv[1] = t1.to(torch.float32)
    return dict(left=torch.stack(L), right=torch.stack(Rimg), disp=torch.stack(D), R=Rm, t=tv,
                K=rig.K(), baseline=rig.baseline, rig=rig, max_disp=64)


def kitti_like_sequence(seed: int, n_frames: int = 100, width: int = 1242, height: int = 375,
                        f: float = 721.0, baseline: float = 0.54, n_boxes: int = 20, n_moving: int = 3,
                        device="cpu", render_frames: int | None = None):
    """A drive through a box-lined scene shaped like a KITTI raw sequence.

    Ego-motion: about 1 m/frame forward with a smooth yaw (at most 1 degree per
    frame).  Scene: ground plane (camera 1.65 m above it), a backdrop far enough
    that every disparity is >= 1, and n_boxes boxes on the ground, n_moving of
    which move on their own at 0.5-2 m/frame along the road.  Box faces stay at
    least 4 m beside the path so that disparities stay below 128.  Only the
    first ``render_frames`` frames (default: all) are rendered; the scene and
    motion are those of the n_frames-long sequence either way.
    """
    g = torch.Generator().manual_seed(seed)

    def u(a, b):
        return a + (b - a) * torch.rand((), generator=g).item()

    rig = Rig(width, height, f, baseline)
    amp = math.radians(u(2.0, 4.0))
    period = u(40.0, 80.0)
    phase = u(0.0, 2 * math.pi)
    # camera poses
    Rs, cs = [], []
    psi = 0.0
    pos = torch.zeros(3, dtype=torch.float64)
    psis = []
    for k in range(n_frames):
        psi_k = amp * math.sin(2 * math.pi * k / period + phase) - amp * math.sin(phase)
        psi_k += math.radians(u(-0.1, 0.1))
        if k > 0:
            step = u(0.9, 1.1)
            heading = psis[-1]
            pos = pos + torch.tensor([math.sin(heading) * step, 0.0, math.cos(heading) * step],
                                     dtype=torch.float64)
        psis.append(psi_k)
        Rs.append(_yaw(psi_k))
        cs.append(pos.clone())
    path_z = torch.stack(cs)[:, 2].contiguous()
    path_x = torch.stack(cs)[:, 0].contiguous()

    def path_x_at(z):
        i = int(torch.clamp(torch.searchsorted(path_z, torch.tensor(float(z), dtype=torch.float64)), 0, n_frames - 1))
        return float(path_x[i])

    ground_y = 1.65
    zmax = float(path_z[-1]) + 70.0
    boxes = []
    for bi in range(n_boxes):
        moving = bi < n_moving
        side = 1 if torch.rand((), generator=g).item() < 0.5 else -1
        if moving:
            hx, hy, hz = 0.9, 0.75, 2.0
            z = u(15.0, 45.0)
            gap = u(4.0, 8.0)
            speed = u(0.5, 2.0) * (1 if torch.rand((), generator=g).item() < 0.5 else -1)
            vel = (0.0, 0.0, speed)
        else:
            hx, hy, hz = u(0.5, 2.0), u(0.5, 1.75), u(0.5, 2.0)
            z = u(8.0, zmax)
            gap = u(4.0, 14.0)
            vel = (0.0, 0.0, 0.0)
        x = path_x_at(z) + side * (gap + hx)
        boxes.append(Box((x, ground_y - hy, z), (hx, hy, hz), vel, texel=u(0.04, 0.08)))
    wall_z = f * baseline / 1.1       # disparity 1.1 at frame 0, larger afterwards
    scene = Scene(seed=seed, ground_y=ground_y, wall_z=wall_z, boxes=boxes, ground_texel=0.05,
                  wall_texel=0.6)
    ngen = torch.Generator(device=device).manual_seed(seed + 7919)
    H, W = height, width
    nr = n_frames if render_frames is None else min(render_frames, n_frames)
    left = torch.empty(nr, H, W, dtype=torch.uint8, device=device)
    right = torch.empty_like(left)
    disp = torch.empty(nr, H, W, dtype=torch.float32, device=device)
    Rm = torch.zeros(nr, 3, 3, dtype=torch.float32)
    tv = torch.zeros(nr, 3, dtype=torch.float32)
    Rm[0] = torch.eye(3)
    for k in range(nr):
        l, r, d = render(scene, rig, Rs[k], cs[k], k, 2.0, ngen, device)
        left[k], right[k], disp[k] = l, r, d
        if k > 0:
            R1, t1 = relative_motion(Rs[k - 1], cs[k - 1], Rs[k], cs[k])
            Rm[k] = R1.to(torch.float32)
            tv[k] = t1.to(torch.float32)
    return dict(left=left, right=right, disp=disp, R=Rm, t=tv, K=rig.K(), baseline=baseline, rig=rig,
                max_disp=128)


def network_params(seed: int, layers=((4, 32), (32, 32), (32, 32), (32, 6))):
    """Seeded initial parameters of a stack of 3x3 layers: He-normal weights
    (std sqrt(2 / (9 in))) and zero biases, flat float32, layer by layer with
    the weights in (out, in, ky, kx) order followed by the bias."""
    import numpy as np
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in layers:
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (ci * 9)), co * ci * 9))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)
