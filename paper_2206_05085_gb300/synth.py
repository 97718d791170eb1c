"""Seeded synthetic inputs for the volume-rendering training step.

This module only draws random numbers and lays them out: density and feature
grids built from Gaussian blobs, camera rays, target colours and the initial
weights of the colour MLP and of the proposal MLP.  It holds none of the
method's arithmetic (no alpha, no compositing, no sampling along rays); both
the CUDA path and the CPU oracle consume what it returns.

The paper's datasets (Synthetic-NeRF, Tanks&Temples, LLFF, mip-NeRF 360) are
not available, so scenes of the same grid sizes and sample counts stand in
for them (Sec. 5: 160^3 bounded grids, 320^3 unbounded grids).

Every array comes from numpy's PCG64 seeded by ``seed``; each array draws
from its own child stream of ``SeedSequence(seed)`` in a fixed order, so
adding an array never changes the others.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Child-stream slots (fixed order; never renumber).
_S_BLOB, _S_NOISE, _S_FEAT, _S_RAY_O, _S_RAY_J, _S_TARGET, _S_MLP, _S_PROP, _S_SHELL, _S_DETAIL = range(10)


def _streams(seed: int, n: int = 16):
    return [np.random.Generator(np.random.PCG64(s)) for s in np.random.SeedSequence(seed).spawn(n)]


@dataclasses.dataclass
class SceneConfig:
    """Shape of one synthetic workload.

    bbox_min/bbox_max: world (or contracted-space) box covered by the grids.
    grid: grid points per axis (corner aligned, so voxel size is
    extent / (grid - 1)).  n_blobs/sigma_lo/sigma_hi/blob_peak/blob_bias/
    noise_std: density recipe D(x) = bias + (peak - bias) sum_b
    exp(-|x-c_b|^2/(2 sigma_b^2)) + N(0, noise_std^2), so an isolated blob
    reaches raw = peak at its centre.  feat_dim/feat_std: feature grid
    N(0, std^2).
    """

    name: str
    grid: int
    bbox_min: float
    bbox_max: float
    n_rays: int
    n_blobs: int
    sigma_lo: float
    sigma_hi: float
    blob_peak: float = 10.0
    blob_bias: float = -4.0
    noise_std: float = 0.1
    feat_dim: int = 12
    feat_std: float = 0.1
    blob_center_range: float = 1.0
    camera: str = "sphere"          # "sphere" (radius cam_radius), "circle" (z=0, radius cam_radius)
                                    # or "forward" (pinhole cameras near z=0 looking down -z)
    cam_radius: float = 4.0
    jitter: float = 0.3
    shell: tuple | None = None      # (r_lo, r_hi, raw) background shell in contracted L-inf radius
    dims: tuple | None = None       # (Gx, Gy, Gz) when the grid is not cubic
    focal: float = 400.0            # "forward": pinhole focal length and image size (pixels)
    img_w: int = 400
    img_h: int = 400


CFG1 = SceneConfig("small_64", grid=64, bbox_min=-2.0, bbox_max=2.0, n_rays=2048,
                   n_blobs=3, sigma_lo=0.2, sigma_hi=0.5)
CFG2 = SceneConfig("dvgo_160", grid=160, bbox_min=-1.0, bbox_max=1.0, n_rays=8192,
                   n_blobs=10, sigma_lo=0.12, sigma_hi=0.25, blob_center_range=0.5,
                   jitter=0.15)
CFG3 = SceneConfig("unbounded_320", grid=320, bbox_min=-2.0, bbox_max=2.0, n_rays=8192,
                   n_blobs=20, sigma_lo=0.05, sigma_hi=0.2, blob_center_range=0.6,
                   camera="circle", cam_radius=1.0, shell=(1.6, 1.9, 6.0))
CFG4 = dataclasses.replace(CFG2, name="dvgo_160_bf16", n_rays=16384)
CFG5 = dataclasses.replace(CFG2, name="dvgo_160_proposal", n_rays=16384)
# Forward-facing capture (Sec. 5.3): the grid lives in normalized device
# coordinates, D = 256 depth layers of 384 x 384 (multiplane-image layout).
CFG6 = SceneConfig("forward_facing_384", grid=384, dims=(384, 384, 256), bbox_min=-1.0, bbox_max=1.0,
                   n_rays=8192, n_blobs=24, sigma_lo=0.12, sigma_hi=0.3, blob_center_range=0.7,
                   camera="forward", cam_radius=0.1, jitter=0.0)

CONFIGS = {c.name: c for c in (CFG1, CFG2, CFG3, CFG4, CFG5, CFG6)}


def grid_dims(cfg: SceneConfig) -> tuple:
    """Grid points per axis (x, y, z)."""
    return tuple(cfg.dims) if cfg.dims is not None else (cfg.grid,) * 3


def grid_axis(cfg: SceneConfig, axis: int = 0) -> np.ndarray:
    return np.linspace(cfg.bbox_min, cfg.bbox_max, grid_dims(cfg)[axis], dtype=np.float64)


def density_grid(cfg: SceneConfig, seed: int = 0) -> np.ndarray:
    """Raw density at the grid points, float32, dense [Z][Y][X] (x fastest)."""
    st = _streams(seed)
    rb = st[_S_BLOB]
    c = rb.uniform(-cfg.blob_center_range, cfg.blob_center_range, (cfg.n_blobs, 3))
    s = rb.uniform(cfg.sigma_lo, cfg.sigma_hi, cfg.n_blobs)
    Z, Y, X = np.meshgrid(grid_axis(cfg, 2), grid_axis(cfg, 1), grid_axis(cfg, 0), indexing="ij")
    D = np.full(X.shape, cfg.blob_bias, dtype=np.float64)
    amp = cfg.blob_peak - cfg.blob_bias      # an isolated blob peaks at blob_peak
    for b in range(cfg.n_blobs):
        r2 = (X - c[b, 0]) ** 2 + (Y - c[b, 1]) ** 2 + (Z - c[b, 2]) ** 2
        D += amp * np.exp(-r2 / (2.0 * s[b] ** 2))
    if cfg.shell is not None:
        r_lo, r_hi, val = cfg.shell
        rinf = np.maximum(np.maximum(np.abs(X), np.abs(Y)), np.abs(Z))
        D = np.where((rinf >= r_lo) & (rinf <= r_hi), np.maximum(D, val), D)
    D += st[_S_NOISE].normal(0.0, cfg.noise_std, D.shape)
    return np.ascontiguousarray(D.astype(np.float32))


def feature_grid(cfg: SceneConfig, seed: int = 0) -> np.ndarray:
    """Feature grid, float32, dense [Z][Y][X][C] (channel innermost)."""
    st = _streams(seed)
    gx, gy, gz = grid_dims(cfg)
    return np.ascontiguousarray(
        st[_S_FEAT].normal(0.0, cfg.feat_std, (gz, gy, gx, cfg.feat_dim)).astype(np.float32))


def _orthonormal_pair(d: np.ndarray):
    a = np.where(np.abs(d[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    u = np.cross(d, a)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = np.cross(d, u)
    return u, v


def _rotate(vec, axis, ang):
    # Rodrigues rotation of vec about unit axis by ang (radians).
    c, s = np.cos(ang)[:, None], np.sin(ang)[:, None]
    return vec * c + np.cross(axis, vec) * s + axis * np.sum(axis * vec, 1, keepdims=True) * (1 - c)


def rays(cfg: SceneConfig, seed: int = 0, n_rays: int | None = None):
    """Ray origins and unit directions, float32 [R,3] each.

    "sphere": origins uniform on a sphere of radius cam_radius, aimed at the
    origin; "circle": origins on the circle of radius cam_radius in z=0.
    Each direction is then rotated by two angles U[-jitter, jitter] about two
    axes orthogonal to it.  "forward": pinhole cameras with centres uniform in
    the disc of radius cam_radius in z = 0, all looking down -z; each ray goes
    through a pixel (u, v) uniform over the img_w x img_h image, direction
    ((u - w/2)/f, -(v - h/2)/f, -1) normalised.
    """
    R = cfg.n_rays if n_rays is None else n_rays
    st = _streams(seed)
    ro = st[_S_RAY_O]
    if cfg.camera == "forward":
        rr = cfg.cam_radius * np.sqrt(ro.uniform(0, 1, R))
        phi = ro.uniform(0, 2 * math.pi, R)
        o = np.stack([rr * np.cos(phi), rr * np.sin(phi), np.zeros(R)], 1)
        rj = st[_S_RAY_J]
        u = rj.uniform(0, cfg.img_w, R)
        v = rj.uniform(0, cfg.img_h, R)
        d = np.stack([(u - 0.5 * cfg.img_w) / cfg.focal, -(v - 0.5 * cfg.img_h) / cfg.focal, -np.ones(R)], 1)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        return (np.ascontiguousarray(o.astype(np.float32)),
                np.ascontiguousarray(d.astype(np.float32)))
    if cfg.camera == "sphere":
        o = ro.normal(size=(R, 3))
        o /= np.linalg.norm(o, axis=1, keepdims=True)
        o *= cfg.cam_radius
    else:
        phi = ro.uniform(0, 2 * math.pi, R)
        o = np.stack([np.cos(phi), np.sin(phi), np.zeros(R)], 1) * cfg.cam_radius
    d = -o / np.linalg.norm(o, axis=1, keepdims=True)
    rj = st[_S_RAY_J]
    a1 = rj.uniform(-cfg.jitter, cfg.jitter, R)
    a2 = rj.uniform(-cfg.jitter, cfg.jitter, R)
    u, v = _orthonormal_pair(d)
    d = _rotate(d, u, a1)
    d = _rotate(d, v, a2)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return (np.ascontiguousarray(o.astype(np.float32)),
            np.ascontiguousarray(d.astype(np.float32)))


def target_rgb(cfg: SceneConfig, seed: int = 0, n_rays: int | None = None) -> np.ndarray:
    R = cfg.n_rays if n_rays is None else n_rays
    return np.ascontiguousarray(_streams(seed)[_S_TARGET].uniform(0, 1, (R, 3)).astype(np.float32))


# Colour MLP (rgbnet): widths 39 -> 128 -> 128 -> 3.  Flat parameter layout,
# float32: W1[128][39], b1[128], W2[128][128], b2[128], W3[3][128], b3[3].
RGBNET_DIMS = (39, 128, 128, 3)
# Proposal MLP: 39 -> 64 -> 64 -> 1, same flat layout.
PROPOSAL_DIMS = (39, 64, 64, 1)


def mlp_num_params(dims) -> int:
    return sum(dims[i + 1] * dims[i] + dims[i + 1] for i in range(len(dims) - 1))


def mlp_params(dims=RGBNET_DIMS, seed: int = 0, slot: int = _S_MLP) -> np.ndarray:
    """Kaiming-uniform initial weights (U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for
    weights and biases), float32 flat vector."""
    rng = _streams(seed)[slot]
    out = []
    for i in range(len(dims) - 1):
        bound = 1.0 / math.sqrt(dims[i])
        out.append(rng.uniform(-bound, bound, dims[i + 1] * dims[i]))
        out.append(rng.uniform(-bound, bound, dims[i + 1]))
    return np.ascontiguousarray(np.concatenate(out).astype(np.float32))


def proposal_params(seed: int = 0) -> np.ndarray:
    return mlp_params(PROPOSAL_DIMS, seed, _S_PROP)


def uniform(shape, lo=0.0, hi=1.0, seed: int = 0, stream: int = 15, dtype=np.float32):
    """Generic seeded uniform array (test inputs such as upstream gradients)."""
    return np.ascontiguousarray(_streams(seed)[stream].uniform(lo, hi, shape).astype(dtype))


def normal(shape, std=1.0, seed: int = 0, stream: int = 14, dtype=np.float32):
    return np.ascontiguousarray(_streams(seed)[stream].normal(0.0, std, shape).astype(dtype))


def truth_detail(shape, std: float, seed: int = 0) -> np.ndarray:
    """Fine-scale detail of the held-out truth scene: i.i.d. N(0, std^2),
    float32, drawn in float32 (the arrays are large)."""
    rng = _streams(seed)[_S_DETAIL]
    out = rng.standard_normal(shape, dtype=np.float32)
    out *= np.float32(std)
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float32.  This is a storage format conversion, used so that both sides can
    read the same BF16-stored parameters."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    r = r.astype(np.uint32)
    nan = np.isnan(x)
    out = r.view(np.float32).copy()
    out[nan] = np.nan
    return out


@dataclasses.dataclass
class RenderParams:
    """Hyper-parameters of one workload, passed unchanged to both sides.

    Sampling: t_k = t_lo + (k + step_offset) * step for k < max_steps, where
    [t_lo, t_hi] is [near, far], clipped to the ray's bbox slab when
    use_slab.  Contracted workloads march with a contracted-space step
    (step_c) instead.  interval: the alpha interval in voxel units.
    """

    near: float
    far: float
    step: float
    step_offset: float
    use_slab: bool
    max_steps: int
    interval: float
    alpha_init: float = 1e-4
    T_stop: float = 1e-3
    bg: tuple = (1.0, 1.0, 1.0)
    lambda_dist: float = 0.01
    tv_w_density: float = 0.0
    tv_w_feature: float = 0.0
    tv_delta: float = 1.0
    mask_thres: float | None = None     # occupancy mask alpha threshold (None: no mask)
    contracted: bool = False
    ndc: bool = False               # forward-facing: NDC warp, samples on the depth layers
    ndc_fx: float = 0.0             # focal / (img_w / 2)
    ndc_fy: float = 0.0             # focal / (img_h / 2)
    ndc_near: float = 1.0
    contract_b: float = 1.0
    contract_p_inf: bool = True
    step_c: float = 0.0
    lr_grid: float = 0.1
    lr_mlp: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.99
    eps: float = 1e-15


def voxel_size(cfg: SceneConfig) -> np.float32:
    return np.float32((cfg.bbox_max - cfg.bbox_min) / (cfg.grid - 1))


def render_params(cfg: SceneConfig) -> RenderParams:
    if cfg.camera == "forward":
        # Sec. 5.3 implementation details: step of one layer, TV weights 1e-5
        # (density) and 1e-6 (features), distortion weight 1e-2; the alpha
        # interval is the step in voxel (layer) units
        D = grid_dims(cfg)[2]
        return RenderParams(near=0.0, far=0.0, step=1.0, step_offset=0.0, use_slab=False, max_steps=D,
                            interval=1.0, tv_w_density=1e-5, tv_w_feature=1e-6, mask_thres=1e-4,
                            ndc=True, ndc_fx=float(np.float32(cfg.focal / (0.5 * cfg.img_w))),
                            ndc_fy=float(np.float32(cfg.focal / (0.5 * cfg.img_h))), ndc_near=1.0)
    vs = voxel_size(cfg)
    if cfg.grid == 64:
        step = np.float32(4.0 / 128)
        return RenderParams(near=2.0, far=6.0, step=float(step), step_offset=0.5,
                            use_slab=False, max_steps=128, interval=float(step / vs))
    if cfg.camera == "circle":
        step_c = np.float32(np.float32(0.5) * vs)
        return RenderParams(near=0.0, far=0.0, step=0.0, step_offset=0.5, use_slab=False,
                            max_steps=512, interval=0.5, bg=(0.0, 0.0, 0.0),
                            tv_w_density=1e-6, tv_w_feature=1e-7, contracted=True,
                            contract_b=1.0, contract_p_inf=True, step_c=float(step_c))
    step = np.float32(np.float32(0.5) * vs)
    diag = math.sqrt(3.0) * (cfg.bbox_max - cfg.bbox_min)
    return RenderParams(near=0.0, far=1.0e4, step=float(step), step_offset=0.0, use_slab=True,
                        max_steps=int(math.ceil(diag / float(step))) + 8, interval=0.5,
                        tv_w_density=1e-6, tv_w_feature=1e-7, mask_thres=1e-4)
