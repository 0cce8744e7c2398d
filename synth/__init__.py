"""Seeded synthetic point clouds and fields shaped like the paper's workloads.

The paper measures on meshes (Thingi10K, the Alien/Duck/Land/Octocat meshes,
flag_simple) that are not available here; these generators stand in for them
with surfaces in R^3 of the same sizes (up to ~1.5M nodes, Sec. 3.1), 3-channel
and wider fields (Sec. 3.1, vertex normals / velocities), and eps, lambda at the
paper's scale (Sec. 3.2, App. D.1.3, App. E).

This module holds NO arithmetic of the RFD method: it only draws inputs
(points, fields, per-cloud parameters).  Both the CUDA path and the CPU oracle
consume what it returns; neither shares any other code.

Every draw uses numpy's PCG64 generator keyed by (seed, stream) so the same
call always returns the same arrays.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "rng_for", "unit_sphere", "torus", "ellipsoid_union", "gaussian_field",
    "CloudSpec", "config_single", "batched_specs", "serving_trace", "make_cloud", "gw_problem", "eigen_specs",
]

# stream ids keep the points, the field and the per-cloud parameters independent
_STREAM_POINTS = 1
_STREAM_FIELD = 2
_STREAM_PARAMS = 3
_STREAM_ARRIVALS = 4
_STREAM_GW = 5


def rng_for(seed: int, stream: int, sub: int = 0) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream), int(sub)])


def unit_sphere(n: int, rng: np.random.Generator, radius: float = 1.0) -> np.ndarray:
    """Uniform on the sphere of the given radius: normalised Gaussian vectors."""
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return (radius * g).astype(np.float32)


def torus(n: int, rng: np.random.Generator, R: float = 1.0, r: float = 0.3,
          jitter: float = 0.0) -> np.ndarray:
    """Area-uniform torus surface (tube radius r around a circle of radius R).

    The tube angle v is accepted with probability (R + r cos v)/(R + r), the
    area element's relative size; then optional N(0, jitter^2) per coordinate.
    """
    out = np.empty((0, 2))
    while out.shape[0] < n:
        k = 2 * (n - out.shape[0]) + 64
        v = rng.uniform(0.0, 2 * np.pi, k)
        acc = rng.uniform(0.0, 1.0, k) < (R + r * np.cos(v)) / (R + r)
        u = rng.uniform(0.0, 2 * np.pi, k)
        out = np.concatenate([out, np.stack([u[acc], v[acc]], 1)])
    u, v = out[:n, 0], out[:n, 1]
    p = np.stack([(R + r * np.cos(v)) * np.cos(u),
                  (R + r * np.cos(v)) * np.sin(u),
                  r * np.sin(v)], 1)
    if jitter > 0:
        p = p + rng.normal(0.0, jitter, p.shape)
    return p.astype(np.float32)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, rr = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(rr))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _ellipsoid(n: int, rng: np.random.Generator, axes: np.ndarray) -> np.ndarray:
    """Area-uniform ellipsoid surface with the given semi-axes (centred, unrotated).

    A unit direction u mapped to diag(axes) u has area density proportional to
    sqrt(sum u_i^2 / a_i^2); accept with that density times min(axes) <= 1.
    """
    out = np.empty((0, 3))
    while out.shape[0] < n:
        k = 2 * (n - out.shape[0]) + 64
        u = rng.standard_normal((k, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        dens = np.sqrt(((u / axes[None, :]) ** 2).sum(1)) * axes.min()
        acc = rng.uniform(0.0, 1.0, k) < dens
        out = np.concatenate([out, u[acc]])
    return out[:n] * axes[None, :]


def ellipsoid_union(n: int, rng: np.random.Generator, k: int = 8) -> np.ndarray:
    """Union of k random ellipsoid surfaces, n/k points each.

    Semi-axes U[0.2, 1], a random rotation (sign-fixed QR of a Gaussian 3x3),
    centres U[0, 1]^3 (the ellipsoids may extend outside the unit cube).
    """
    per = [n // k + (1 if i < n % k else 0) for i in range(k)]
    parts = []
    for i in range(k):
        axes = rng.uniform(0.2, 1.0, 3)
        rot = _random_rotation(rng)
        centre = rng.uniform(0.0, 1.0, 3)
        parts.append(_ellipsoid(per[i], rng, axes) @ rot.T + centre[None, :])
    return np.concatenate(parts).astype(np.float32)


def gaussian_field(n: int, c: int, seed: int, sub: int = 0) -> np.ndarray:
    """F in R^{n x c}, i.i.d. N(0, 1), float32, from its own stream."""
    return rng_for(seed, _STREAM_FIELD, sub).standard_normal((n, c)).astype(np.float32)


@dataclasses.dataclass
class CloudSpec:
    """One GFI problem: a point cloud plus the RFD parameters (eps, lambda, m)."""
    kind: str          # "sphere" | "torus" | "ellipsoids"
    n: int
    m: int
    c: int
    eps: float
    lam: float
    seed: int          # seed of the random features (omega) and of the field
    scale: float = 1.0
    jitter: float = 0.0
    sub: int = 0       # sub-stream of the point draws
    field_sub: int = -1  # sub-stream of the field draw (-1: same as `sub`)


def make_cloud(spec: CloudSpec) -> tuple[np.ndarray, np.ndarray]:
    """(points N x 3 float32, F N x c float32) for a spec."""
    rng = rng_for(spec.seed, _STREAM_POINTS, spec.sub)
    if spec.kind == "sphere":
        pts = unit_sphere(spec.n, rng, spec.scale)
    elif spec.kind == "torus":
        pts = torus(spec.n, rng, R=spec.scale, r=0.3 * spec.scale, jitter=spec.jitter)
    elif spec.kind == "ellipsoids":
        pts = ellipsoid_union(spec.n, rng, 8)
    else:
        raise ValueError(spec.kind)
    fsub = spec.sub if spec.field_sub < 0 else spec.field_sub
    return pts, gaussian_field(spec.n, spec.c, spec.seed, fsub)


def config_single(name: str, c: int | None = None) -> CloudSpec:
    """The single-cloud workloads.

    small   : N=2,048 on the unit sphere, eps=0.1, lambda=0.1, m=64, c=3
    torus   : N=100,000 on a torus (R=1, r=0.3, jitter 0.005), eps=lambda=0.05, m=256, c=16
    large   : N=1,000,000 on 8 ellipsoids, eps=lambda=0.02, m=1024, c=3 (or 64)
    tiny    : N=256 on the unit sphere (brute-force exact exp(lambda W)F check)
    """
    if name == "small":
        return CloudSpec("sphere", 2048, 64, c or 3, 0.1, 0.1, 0)
    if name == "tiny":
        return CloudSpec("sphere", 256, 64, c or 3, 0.1, 0.1, 0)
    if name == "torus":
        return CloudSpec("torus", 100_000, 256, c or 16, 0.05, 0.05, 0, scale=1.0, jitter=0.005)
    if name == "large":
        return CloudSpec("ellipsoids", 1_000_000, 1024, c or 3, 0.02, 0.02, 0)
    raise ValueError(name)


def batched_specs(count: int = 512, seed: int = 0, n_lo: float = 1e3, n_hi: float = 2e5,
                  ms=(64, 128, 256), c: int = 8, eps: float = 0.05,
                  lam_lo: float = 0.01, lam_hi: float = 0.2) -> list[CloudSpec]:
    """Many clouds of uneven size: N log-uniform, sphere or torus (50/50) of random
    scale U[0.5, 2], m uniform over `ms`, lambda ~ U[lam_lo, lam_hi]."""
    rng = rng_for(seed, _STREAM_PARAMS)
    specs = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kind = "sphere" if rng.uniform() < 0.5 else "torus"
        scale = float(rng.uniform(0.5, 2.0))
        m = int(ms[rng.integers(0, len(ms))])
        lam = float(rng.uniform(lam_lo, lam_hi))
        specs.append(CloudSpec(kind, n, m, c, eps, lam, seed * 100003 + i, scale=scale, sub=i))
    return specs


def serving_trace(rate: float = 2000.0, duration: float = 10.0, seed: int = 0,
                  n_lo: float = 500, n_hi: float = 5e5, reuse: float = 0.3,
                  eps: float = 0.05, lam_lo: float = 0.01, lam_hi: float = 0.2,
                  max_requests: int | None = None):
    """Poisson arrivals of GFI requests.

    Returns a list of (t_arrival_s, CloudSpec, reuse_of) where reuse_of is the
    index of an earlier request whose cloud (points, m, eps, lambda, omega) is
    reused with a new field, or -1 for a new cloud.  N log-uniform in
    [n_lo, n_hi], m in {64, ..., 512} step 64, c in 1..32.
    """
    rng = rng_for(seed, _STREAM_ARRIVALS)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration or (max_requests is not None and len(out) >= max_requests):
            break
        i = len(out)
        c = int(rng.integers(1, 33))
        if out and rng.uniform() < reuse:
            j = int(rng.integers(0, len(out)))
            while out[j][2] >= 0:
                j = out[j][2]
            base = out[j][1]
            spec = dataclasses.replace(base, c=c, field_sub=1_000_000 + i)
            out.append((t, spec, j))
            continue
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kind = "sphere" if rng.uniform() < 0.5 else "torus"
        scale = float(rng.uniform(0.5, 2.0))
        m = int(64 * rng.integers(1, 9))
        lam = float(rng.uniform(lam_lo, lam_hi))
        out.append((t, CloudSpec(kind, n, m, c, eps, lam, seed * 7919 + i, scale=scale, sub=i), -1))
    return out


def gw_problem(n1: int, n2: int, seed: int = 0):
    """Inputs of one (F)GW conditional-gradient iteration between two random 3-D
    point distributions (App. C.2 experiments: uniform in the unit cube).

    Returns (X, Y, T, p, q, Gt, M): clouds X (n1 x 3) and Y (n2 x 3), a positive
    coupling T (n1 x n2, sum 1) with marginals p, q, a second coupling Gt (the
    linearised step's target, so dG = Gt - p q^T) and a feature-cost matrix M
    (distances between random binary node labels, as the FGW experiments do).
    All float64."""
    rng = rng_for(seed, _STREAM_GW)
    X = rng.uniform(0.0, 1.0, (n1, 3))
    Y = rng.uniform(0.0, 1.0, (n2, 3))
    T = rng.uniform(0.0, 1.0, (n1, n2))
    T /= T.sum()
    p, q = T.sum(1), T.sum(0)
    Gt = rng.uniform(0.0, 1.0, (n1, n2))
    Gt /= Gt.sum()
    la, lb = rng.integers(0, 2, n1), rng.integers(0, 2, n2)
    M = (la[:, None] != lb[None, :]).astype(np.float64)
    return X, Y, T, p, q, Gt, M


def eigen_specs(count: int = 1024, seed: int = 0, n: int = 2048, m: int = 64, eps: float = 0.1,
                lam: float = -0.1) -> list[CloudSpec]:
    """Shape-classification clouds (Sec. 3.3: 2048 points sampled per shape,
    eps = 0.1, lambda = -0.1): sphere, torus or ellipsoid union in turn, random
    scale U[0.5, 1] (spheres, tori), one feature seed per cloud; lambda is
    the raw value (callers apply their units)."""
    rng = rng_for(seed, _STREAM_PARAMS, 1)
    kinds = ("sphere", "torus", "ellipsoids")
    return [CloudSpec(kinds[i % 3], n, m, 1, eps, lam, seed * 100003 + i, scale=float(rng.uniform(0.5, 1.0)), sub=i)
            for i in range(count)]
