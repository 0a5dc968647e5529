"""Seeded synthetic inputs for the neural radiance cache hot path.

This module holds no arithmetic of the method (no encoding, network, loss or
optimiser).  It only draws the inputs that both the FP64 oracle and the CUDA
path consume, so that both sides see bit-identical FP32 values:

* query / training records in the 64-byte boundary layout
  ``[x0,x1,x2, u_w,v_w, u_n,v_n, r, a0,a1,a2, b0,b1,b2, 0,0]``
  (x in [0,1]^3; direction and normal as spherical coordinates normalised to
  [0,1]^2, i.e. (theta/pi, phi/(2 pi)) as in Table 1's caption; roughness and
  the two albedos uniform in [0,1]);
* Xavier-uniform initial weights;
* training targets from a seeded analytic HDR radiance field (a sum of eight
  anisotropic Gaussians in position times cosine lobes in direction with
  log-normal RGB amplitudes).  The field stands in for the path tracer's
  radiance estimates, which the paper gathers along training paths (Sec. 3.5).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then the variant-13 finaliser.  Stream ``s`` of base seed ``b`` starts from
state ``b * 0x100000001B3 + s`` (mod 2^64).  A uniform double in [0,1) is the
top 53 bits of an output times 2^-53.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
REC_FLOATS = 16  # 64-byte record

STREAM_RECORDS = 1
STREAM_WEIGHTS = 2
STREAM_FIELD = 3
STREAM_FRAMES = 4
BASE_SEED = 2106


def splitmix64_next(state: int) -> tuple[int, int]:
    """One SplitMix64 step on a Python int: returns (new_state, output)."""
    state = (state + GOLDEN_GAMMA) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def splitmix64_array(state0: int, count: int) -> np.ndarray:
    """The first ``count`` SplitMix64 outputs from ``state0`` (vectorised)."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(state0 & MASK64) + idx * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def stream_state(base_seed: int, stream: int) -> int:
    return (base_seed * 0x100000001B3 + stream) & MASK64


def uniforms(base_seed: int, stream: int, count: int, skip: int = 0) -> np.ndarray:
    """``count`` uniform doubles in [0,1) from stream ``stream``, after ``skip`` draws."""
    state = (stream_state(base_seed, stream) + skip * GOLDEN_GAMMA) & MASK64
    z = splitmix64_array(state, count)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def make_records(n: int, seed: int = BASE_SEED, stream: int = STREAM_RECORDS) -> np.ndarray:
    """``n`` query records, float32 [n, 16], drawn from the paper-shaped distribution.

    Directions and normals are uniform on the sphere: theta = arccos(1 - 2u),
    phi = 2 pi v, stored normalised as (theta/pi, phi/(2 pi)).
    """
    u = uniforms(seed, stream, 14 * n).reshape(n, 14) if n > 0 else np.zeros((0, 14))
    rec = np.zeros((n, REC_FLOATS), dtype=np.float64)
    rec[:, 0:3] = u[:, 0:3]
    rec[:, 3] = np.arccos(1.0 - 2.0 * u[:, 3]) / math.pi
    rec[:, 4] = u[:, 4]
    rec[:, 5] = np.arccos(1.0 - 2.0 * u[:, 5]) / math.pi
    rec[:, 6] = u[:, 6]
    rec[:, 7] = u[:, 7]
    rec[:, 8:14] = u[:, 8:14]
    return rec.astype(np.float32)


def layer_dims(width: int = 64, hidden_layers: int = 5, in_dims: int = 64, out_dims: int = 3) -> list[int]:
    """Neuron counts d_0..d_L: encoded input, ``hidden_layers`` hidden layers, RGB output."""
    return [in_dims] + [width] * hidden_layers + [out_dims]


def n_params(dims: list[int]) -> int:
    return sum(dims[i + 1] * dims[i] for i in range(len(dims) - 1))


def xavier_weights(dims: list[int], seed: int = BASE_SEED, stream: int = STREAM_WEIGHTS) -> np.ndarray:
    """Flat float32 weights, layer after layer, each row-major [out][in].

    Layer l draws U(-a, a) with a = sqrt(6 / (fan_in + fan_out)) (Glorot &
    Bengio 2010), computed in FP64 and rounded to FP32.
    """
    total = n_params(dims)
    u = uniforms(seed, stream, total)
    out = np.empty(total, dtype=np.float64)
    off = 0
    for i in range(len(dims) - 1):
        fan_in, fan_out = dims[i], dims[i + 1]
        cnt = fan_in * fan_out
        a = math.sqrt(6.0 / (fan_in + fan_out))
        out[off:off + cnt] = (2.0 * u[off:off + cnt] - 1.0) * a
        off += cnt
    return out.astype(np.float32)


def _box_muller(u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


class RadianceField:
    """Seeded analytic HDR radiance field L(x, w), 8 lobes, RGB.

    L(x, w) = sum_g A_g * exp(-1/2 sum_j ((x_j - mu_gj) / s_gj)^2) * max(0, w . d_g)^e_g
    with mu ~ U[0,1]^3, s ~ U[0.05, 0.3]^3, A_g = exp(N(0,1)) per channel,
    d_g uniform on the sphere, e_g ~ U[1, 16].
    """

    G = 8

    def __init__(self, seed: int = BASE_SEED, stream: int = STREAM_FIELD):
        u = uniforms(seed, stream, self.G * 15).reshape(self.G, 15)
        self.mu = u[:, 0:3]
        self.s = 0.05 + 0.25 * u[:, 3:6]
        self.amp = np.exp(_box_muller(u[:, 6:9], u[:, 9:12]))
        z = 1.0 - 2.0 * u[:, 12]
        phi = 2.0 * math.pi * u[:, 13]
        rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        self.d = np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)
        self.e = 1.0 + 15.0 * u[:, 14]

    def __call__(self, rec: np.ndarray) -> np.ndarray:
        """Targets float32 [n, 3] for records [n, 16] (FP32 inputs promoted to FP64)."""
        r = rec.astype(np.float64)
        x = r[:, 0:3]
        theta = r[:, 3] * math.pi
        phi = r[:, 4] * 2.0 * math.pi
        w = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)
        out = np.zeros((r.shape[0], 3))
        for g in range(self.G):
            q = ((x - self.mu[g]) / self.s[g]) ** 2
            spatial = np.exp(-0.5 * q.sum(axis=1))
            lobe = np.maximum(0.0, w @ self.d[g]) ** self.e[g]
            out += (spatial * lobe)[:, None] * self.amp[g][None, :]
        return out.astype(np.float32)


def make_training_pool(n: int, seed: int = BASE_SEED) -> tuple[np.ndarray, np.ndarray]:
    """A frame's training-record pool: records [n,16] and their targets [n,3]."""
    rec = make_records(n, seed=seed, stream=STREAM_RECORDS + 16)
    return rec, RadianceField(seed)(rec)


def frame_seed(base_seed: int, frame: int) -> int:
    """The 64-bit seed of frame ``frame`` (drives the training-record shuffle)."""
    _, out = splitmix64_next((stream_state(base_seed, STREAM_FRAMES) + frame * GOLDEN_GAMMA) & MASK64)
    return out


# ------------------------------------------------------------ synthetic paths
# Stand-in for the path tracer that produces the cache's queries and training
# records: cosine-sampled random walks inside the unit cube [0,1]^3 (inward
# normals) seen from a pinhole camera, with an emissive patch on the ceiling.
# Per vertex the generator records what a path tracer knows there.  It draws
# with numpy's PCG64 (O'Neill 2014) and holds none of the method's arithmetic:
# termination, transport and record assembly are the method's steps and live
# in the kernels (and, independently, in the oracle).
PATH_VERTEX_FLOATS = 24
# layout of one vertex (float32): 0-2 position, 3-4 direction towards the
# previous vertex and 5-6 normal (both as (theta/pi, phi/(2 pi))), 7 roughness,
# 8-10 diffuse albedo, 11-13 specular albedo (0-13: the query record's first 14
# floats), 14 pdf (solid angle) of the direction that reached this vertex, 15
# |cos| between that direction and the normal here, 16-18 emitted radiance,
# 19-21 throughput weight of the bounce leaving this vertex (BSDF cos / pdf),
# 22 a uniform for Russian roulette, 23 zero.
PATH_CAMERA = (0.5, 0.5, 0.02)


def _spherical01(d: np.ndarray) -> np.ndarray:
    theta = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    phi = np.mod(np.arctan2(d[:, 1], d[:, 0]), 2.0 * math.pi)
    return np.stack([theta / math.pi, phi / (2.0 * math.pi)], axis=1)


def _cube_hit(o: np.ndarray, d: np.ndarray):
    """First wall of the unit cube hit from inside: point, axis, inward normal."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(d > 0, (1.0 - o) / d, np.where(d < 0, -o / d, np.inf))
    axis = np.argmin(t, axis=1)
    tm = t[np.arange(len(o)), axis]
    x = np.clip(o + tm[:, None] * d, 0.0, 1.0)
    nrm = np.zeros_like(o)
    nrm[np.arange(len(o)), axis] = -np.sign(d[np.arange(len(o)), axis])
    return x, axis, nrm


def make_paths(width: int, height: int, n_vertices: int = 10, seed: int = BASE_SEED) -> np.ndarray:
    """Paths of a width x height viewport: float32 [height*width, n_vertices, 24] (row-major pixels)."""
    rng = np.random.default_rng(seed)
    P = width * height
    cam = np.array(PATH_CAMERA)
    py, px = np.divmod(np.arange(P), width)
    tan = math.tan(math.radians(35.0))
    d = np.stack([((px + 0.5) / width - 0.5) * 2 * tan * width / height, ((py + 0.5) / height - 0.5) * 2 * tan,
                  np.ones(P)], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.repeat(cam[None, :], P, axis=0)
    out = np.zeros((P, n_vertices, PATH_VERTEX_FLOATS), dtype=np.float64)
    pdf_in = np.ones(P)
    for k in range(n_vertices):
        x, axis, nrm = _cube_hit(o, d)
        out[:, k, 0:3] = x
        out[:, k, 3:5] = _spherical01(-d)
        out[:, k, 5:7] = _spherical01(nrm)
        cell = (np.floor(4 * x[:, 0]) + np.floor(4 * x[:, 1]) + np.floor(4 * x[:, 2])) % 2
        albedo = np.where(cell[:, None] > 0, [0.75, 0.62, 0.48], [0.32, 0.42, 0.66]) * (0.7 + 0.1 * axis)[:, None]
        out[:, k, 7] = 0.2 + 0.6 * np.mod(7 * x[:, 0] + 3 * x[:, 1] + 5 * x[:, 2], 1.0)
        out[:, k, 8:11] = albedo
        out[:, k, 11:14] = 0.04
        out[:, k, 14] = pdf_in
        out[:, k, 15] = np.abs(np.sum(d * nrm, axis=1))
        lamp = (axis == 1) & (nrm[:, 1] < 0) & (np.abs(x[:, 0] - 0.5) < 0.2) & (np.abs(x[:, 2] - 0.5) < 0.2)
        out[:, k, 16:19] = np.where(lamp[:, None], [6.0, 6.0, 5.0], 0.0)
        out[:, k, 19:22] = albedo  # Lambertian, cosine-weighted sampling: f cos / pdf = albedo
        out[:, k, 22] = rng.random(P)
        # cosine-weighted direction about the (axis-aligned) normal
        u1, u2 = rng.random(P), rng.random(P)
        r, ph = np.sqrt(u1), 2 * math.pi * u2
        loc = np.stack([r * np.cos(ph), r * np.sin(ph), np.sqrt(np.maximum(0.0, 1.0 - u1))], axis=1)
        t1 = np.zeros_like(nrm)
        t1[np.arange(P), (axis + 1) % 3] = 1.0
        t2 = np.cross(nrm, t1)
        dn = loc[:, 0:1] * t1 + loc[:, 1:2] * t2 + loc[:, 2:3] * nrm
        pdf_in = loc[:, 2] / math.pi
        o = x + 1e-7 * nrm
        d = dn / np.linalg.norm(dn, axis=1, keepdims=True)
    return out.astype(np.float32)
