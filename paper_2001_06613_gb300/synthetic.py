"""Seeded synthetic OCT-like image sequences: the shared input generator.

This module only *produces inputs*.  It holds none of the registration
method's arithmetic (no interpolation, no objective, no predictor): frames are
evaluated in closed form at displaced positions, so the generator never samples
one image grid at another grid's points.

Structure of the stand-in data (the paper's 4D-OCT sequences, Sec. 4 and
Table 1, are not available):

* a layered base image ``B(x)``: bands along the first (depth) axis with
  raised-cosine transitions, like retinal layers;
* Rayleigh-distributed speckle: ``sigma * |Z(x)|`` where ``Z`` is a sum of
  random complex plane waves with speckle-grain wavelengths (6-14 px), so that
  its modulus is Rayleigh(sigma) distributed and it is defined at every point;
* a planted motion ``v_k(x) = sum_j A_j(t_k) c_j sin(2 pi <f_j, x/m> + phi_j)``
  (few low-frequency Fourier modes, temporally smooth amplitudes);
* frames ``R_k(x) = B(x + v_k(x)) + noise``.

Coordinates are in finest-pixel units; the centre of cell ``j`` is ``j + 1/2``
along every axis.  Arrays are C-ordered ``(frame, [component,] axis0, axis1[, axis2])``
and displacement component ``c`` moves along array axis ``c``.
All random draws come from numpy's counter-based Philox generator keyed by the
seed and a stream number.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Sequence, Tuple

import numpy as np

try:  # torch only speeds up the plane-wave sums; numpy gives the same values
    import torch
except Exception:  # pragma: no cover
    torch = None


def philox(seed: int, stream: int) -> np.random.Generator:
    """Counter-based generator for (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


# ---------------------------------------------------------------------------
# workload descriptions
# ---------------------------------------------------------------------------
@dataclass
class SequenceSpec:
    n: int                              # number of frames
    shape: Tuple[int, ...]              # finest grid, C order (depth axis first)
    n_modes: int                        # spatial Fourier modes of the motion
    amp: float                          # max |v| over the whole sequence, px
    periods: Sequence[Tuple[float, float]]   # temporal components: (period, phase)
    noise_sd: float
    speckle_sigma: float = 0.3
    seed: int = 0
    n_waves: int = 48                   # plane waves in the speckle sum

    @property
    def dim(self) -> int:
        return len(self.shape)


def spec_tiny(seed: int = 0) -> SequenceSpec:
    """16 frames of 64x64: 4 modes, 2 px * sin(2 pi t / 16), noise 0.01."""
    return SequenceSpec(n=16, shape=(64, 64), n_modes=4, amp=2.0,
                        periods=[(16.0, 0.0)], noise_sd=0.01, seed=seed)


def spec_paper_scale(seed: int = 1) -> SequenceSpec:
    """200 frames of 256x256: 8 modes, 5 px max, two incommensurate periods."""
    return SequenceSpec(n=200, shape=(256, 256), n_modes=8, amp=5.0,
                        periods=[(37.0, 0.0), (89.0, 0.7)], noise_sd=0.02, seed=seed)


def spec_volume(seed: int = 2) -> SequenceSpec:
    """40 volumes of 128x128x64 (depth first): 6 modes, 4 voxel max, sin(2 pi t/40)."""
    return SequenceSpec(n=40, shape=(64, 128, 128), n_modes=6, amp=4.0,
                        periods=[(40.0, 0.0)], noise_sd=0.01, seed=seed)


def spec_custom(n: int, shape: Sequence[int], seed: int, amp: float = 2.0,
                n_modes: int = 4, noise_sd: float = 0.01) -> SequenceSpec:
    return SequenceSpec(n=n, shape=tuple(int(s) for s in shape), n_modes=n_modes, amp=amp,
                        periods=[(float(max(n, 2)), 0.0)], noise_sd=noise_sd, seed=seed)


# ---------------------------------------------------------------------------
# closed-form ingredients
# ---------------------------------------------------------------------------
def cell_centres(shape: Sequence[int]) -> np.ndarray:
    """(d, *shape) float64 array of finest-grid cell centres (j + 1/2)."""
    axes = [np.arange(s, dtype=np.float64) + 0.5 for s in shape]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=0)


def _raised_cosine_step(t: np.ndarray, width: float) -> np.ndarray:
    s = np.clip((t + 0.5 * width) / width, 0.0, 1.0)
    return 0.5 - 0.5 * np.cos(np.pi * s)


def band_profile(depth: np.ndarray, depth_extent: float) -> np.ndarray:
    """Layered intensity along depth: levels 0.05/0.2/0.6/1.0, edges at 30/55/75 %."""
    levels = (0.05, 0.2, 0.6, 1.0)
    edges = (0.30, 0.55, 0.75)
    out = np.full(depth.shape, levels[0], dtype=np.float64)
    for e, lo, hi in zip(edges, levels[:-1], levels[1:]):
        out += (hi - lo) * _raised_cosine_step(depth - e * depth_extent, 3.0)
    return out


@dataclass
class _Speckle:
    freqs: np.ndarray    # (J, d) rad / px
    coef: np.ndarray     # (J,) complex
    sigma: float

    def __call__(self, pos: np.ndarray, device=None) -> np.ndarray:
        """sigma * |sum_j coef_j exp(i <f_j, pos>)| at positions (d, *S)
        (device: a torch device for the sums, e.g. "cuda"; default the CPU)."""
        d = pos.shape[0]
        flat = pos.reshape(d, -1)
        if torch is not None:
            dev = device or "cpu"
            P = torch.from_numpy(np.ascontiguousarray(flat)).to(dev)
            F = torch.from_numpy(self.freqs).to(dev)
            out = np.empty(flat.shape[1], dtype=np.float64)
            chunk = 1 << 18 if dev == "cpu" else 1 << 22
            cr = torch.from_numpy(self.coef.real.copy()).to(dev)
            ci = torch.from_numpy(self.coef.imag.copy()).to(dev)
            for s in range(0, flat.shape[1], chunk):
                ph = F @ P[:, s:s + chunk]                      # (J, chunk)
                c, sn = torch.cos(ph), torch.sin(ph)
                re = cr @ c - ci @ sn
                im = cr @ sn + ci @ c
                out[s:s + chunk] = torch.sqrt(re * re + im * im).cpu().numpy()
        else:
            ph = self.freqs @ flat
            z = self.coef @ np.exp(1j * ph)
            out = np.abs(z)
        return (self.sigma * out).reshape(pos.shape[1:])


def _make_speckle(spec: SequenceSpec) -> _Speckle:
    g = philox(spec.seed, 1)
    J, d = spec.n_waves, spec.dim
    wavelength = g.uniform(6.0, 14.0, size=J)
    direc = g.normal(size=(J, d))
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    freqs = direc * (2.0 * np.pi / wavelength)[:, None]
    coef = (g.normal(size=J) + 1j * g.normal(size=J)) / math.sqrt(J)
    return _Speckle(freqs=freqs, coef=coef, sigma=spec.speckle_sigma)


@dataclass
class _Motion:
    freqs: np.ndarray      # (M, d) integer cycles per domain
    phases: np.ndarray     # (M,)
    coefs: np.ndarray      # (M, d)
    comp: np.ndarray       # (M,) index of the temporal component driving each mode
    periods: Sequence[Tuple[float, float]]
    shape: Tuple[int, ...]
    scale: float = 1.0

    def temporal(self, t: float) -> np.ndarray:
        return np.array([math.sin(2.0 * math.pi * t / p + ph) for (p, ph) in self.periods])

    def modes(self, pos: np.ndarray) -> List[np.ndarray]:
        """The spatial factors sin(2 pi <f_j, pos / m> + phi_j) of every mode."""
        d = pos.shape[0]
        ext = np.asarray(self.shape, dtype=np.float64).reshape((d,) + (1,) * (pos.ndim - 1))
        return [np.sin(2.0 * np.pi * np.tensordot(self.freqs[j], pos / ext, axes=(0, 0)) + self.phases[j])
                for j in range(self.freqs.shape[0])]

    def from_modes(self, t: float, sines: List[np.ndarray]) -> np.ndarray:
        """v(t, pos) from the spatial factors of :meth:`modes` at pos."""
        d = self.freqs.shape[1]
        a = self.temporal(t)
        out = np.zeros((d,) + sines[0].shape)
        for j, sn in enumerate(sines):
            w = a[self.comp[j]] * sn
            out += self.coefs[j].reshape((d,) + (1,) * sn.ndim) * w[None]
        return self.scale * out

    def __call__(self, t: float, pos: np.ndarray) -> np.ndarray:
        """v(t, pos) for positions (d, *S) -> (d, *S)."""
        return self.from_modes(t, self.modes(pos))


def _make_motion(spec: SequenceSpec) -> _Motion:
    g = philox(spec.seed, 2)
    M, d = spec.n_modes, spec.dim
    freqs = g.integers(1, 3, size=(M, d)).astype(np.float64)
    phases = g.uniform(0, 2 * np.pi, size=M)
    coefs = g.normal(size=(M, d))
    comp = np.arange(M) % len(spec.periods)
    mot = _Motion(freqs, phases, coefs, comp, list(spec.periods), tuple(spec.shape))
    sines = mot.modes(cell_centres(spec.shape))
    peak = 0.0
    for t in range(spec.n):
        v = mot.from_modes(float(t), sines)
        peak = max(peak, float(np.sqrt((v * v).sum(axis=0)).max()))
    mot.scale = spec.amp / peak if peak > 0 else 0.0
    return mot


# ---------------------------------------------------------------------------
# public generator
# ---------------------------------------------------------------------------
def base_image(spec: SequenceSpec, pos: np.ndarray, speckle: _Speckle = None) -> np.ndarray:
    """B(pos) = layered bands(depth) + Rayleigh speckle, pos in px (d, *S)."""
    speckle = speckle or _make_speckle(spec)
    return band_profile(pos[0], float(spec.shape[0])) + speckle(pos)


def make_sequence(spec: SequenceSpec, dtype=np.float32, device=None) -> np.ndarray:
    """Frames R_k(x) = B(x + v_k(x)) + N(0, noise_sd^2), shape (n, *shape)
    (device: torch device for the speckle sums; values equal up to rounding)."""
    speckle = _make_speckle(spec)
    motion = _make_motion(spec)
    x = cell_centres(spec.shape)
    sines = motion.modes(x)
    noise = philox(spec.seed, 3)
    out = np.empty((spec.n,) + tuple(spec.shape), dtype=dtype)
    for k in range(spec.n):
        pos = x + motion.from_modes(float(k), sines)
        img = band_profile(pos[0], float(spec.shape[0])) + speckle(pos, device)
        img += noise.normal(scale=spec.noise_sd, size=img.shape) if spec.noise_sd > 0 else 0.0
        out[k] = img.astype(dtype)
    return out


def planted_motion(spec: SequenceSpec) -> np.ndarray:
    """The planted v_k at the cell centres, shape (n, d, *shape), float64."""
    motion = _make_motion(spec)
    x = cell_centres(spec.shape)
    return np.stack([motion(float(k), x) for k in range(spec.n)], axis=0)


def planted_registration(spec: SequenceSpec, iters: int = 40) -> np.ndarray:
    """Displacements u_k with R_k(x + u_k(x)) = B(x) up to noise.

    They solve ``u_k(x) = -v_k(x + u_k(x))``; the map is a contraction for the
    small, smooth motions generated here, so a fixed-point iteration converges.
    """
    motion = _make_motion(spec)
    x = cell_centres(spec.shape)
    out = np.empty((spec.n, spec.dim) + tuple(spec.shape))
    for k in range(spec.n):
        u = np.zeros_like(x)
        for _ in range(iters):
            u = -motion(float(k), x + u)
        out[k] = u
    return out


def random_field(rng: np.random.Generator, n: int, d: int, shape: Sequence[int],
                 amp: float, rough: float = 0.0, modes: int = 3) -> np.ndarray:
    """Smooth random displacement-like field (n, d, *shape) float32 for parity tests."""
    x = cell_centres(shape)
    ext = np.asarray(shape, dtype=np.float64).reshape((len(shape),) + (1,) * len(shape))
    out = np.zeros((n, d) + tuple(shape))
    for k in range(n):
        for c in range(d):
            acc = np.zeros(tuple(shape))
            for _ in range(modes):
                f = rng.integers(1, 4, size=len(shape)).astype(np.float64)
                acc += rng.normal() * np.sin(2 * np.pi * np.tensordot(f, x / ext, axes=(0, 0))
                                             + rng.uniform(0, 2 * np.pi))
            out[k, c] = amp * acc / modes
    if rough > 0:
        out += rough * rng.normal(size=out.shape)
    return out.astype(np.float32)


# ---------------------------------------------------------------------------
# initial weights of the learned predictor's network (drawn here, passed in)
# ---------------------------------------------------------------------------
NET_CONVS = [(7, 32), (32, 32), (32, 64), (64, 64), (64, 96), (96, 96), (96, 128), (128, 128),
             (224, 96), (96, 96), (160, 64), (64, 64), (96, 32), (32, 32)]


def net_init_params(seed: int, head_scale: float = 0.0) -> np.ndarray:
    """Flat float32 parameter vector of the predictor network: He-normal conv
    weights W[ky][kx][ci][co] (sd sqrt(2 / (9 ci))), zero biases, and a head
    (W[32][2], b[2]) of normal(0, head_scale / sqrt(32)) weights -- zero by
    default, so that the untrained network reproduces linear interpolation."""
    g = philox(seed, 7)
    parts = []
    for ci, co in NET_CONVS:
        parts.append(g.normal(scale=math.sqrt(2.0 / (9 * ci)), size=9 * ci * co))
        parts.append(np.zeros(co))
    parts.append(g.normal(scale=head_scale / math.sqrt(32.0), size=64))
    parts.append(np.zeros(2))
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------------------
# affine-linear motion (the transformations of the paper's experiments, Sec. 4)
# ---------------------------------------------------------------------------
def affine_motion(spec: SequenceSpec, rot_deg: float = 1.5, scale: float = 0.015,
                  shift: float = 1.5) -> Tuple[np.ndarray, np.ndarray]:
    """Planted affine motion about the domain centre c: frame k is sampled at
    x + v_k(x), v_k(x) = (M_k - I)(x - c) + s_k, with M_k a rotation by
    rot_deg sin(2 pi k / n) degrees in the plane of the first two axes scaled by
    1 + scale sin(2 pi k / n + 1), and s_k = shift (sin(2 pi k / n + 2 + i / 2))_i.
    Returns (M (n, d, d), s (n, d))."""
    n, d = spec.n, spec.dim
    M = np.zeros((n, d, d))
    s = np.zeros((n, d))
    for k in range(n):
        ph = 2.0 * math.pi * k / max(n, 1)
        a = math.radians(rot_deg) * math.sin(ph)
        R = np.eye(d)
        R[0, 0], R[0, 1], R[1, 0], R[1, 1] = math.cos(a), -math.sin(a), math.sin(a), math.cos(a)
        M[k] = R * (1.0 + scale * math.sin(ph + 1.0))
        s[k] = [shift * math.sin(ph + 2.0 + 0.5 * i) for i in range(d)]
    return M, s


def blob_image(spec: SequenceSpec, pos: np.ndarray, n_blobs: int = 24, margin: float = 4.0) -> np.ndarray:
    """A smooth image: sum of n_blobs Gaussians of widths 3-6 px at seeded
    centres and heights, times a raised-cosine window that is zero within
    `margin` px of the border and one beyond 3 margin (images on which linear
    interpolation is accurate and zero extension is exact)."""
    g = philox(spec.seed, 4)
    d = pos.shape[0]
    ext = np.asarray(spec.shape, dtype=np.float64)
    out = np.zeros(pos.shape[1:])
    for _ in range(n_blobs):
        mu = g.uniform(0.25, 0.75, size=d) * ext
        sd = g.uniform(3.0, 6.0)
        a = g.uniform(0.5, 1.5)
        r2 = sum((pos[i] - mu[i]) ** 2 for i in range(d))
        out += a * np.exp(-0.5 * r2 / (sd * sd))
    for i in range(d):
        for dist in (pos[i], ext[i] - pos[i]):
            t = np.clip((dist - margin) / (2.0 * margin), 0.0, 1.0)
            out *= 0.5 - 0.5 * np.cos(np.pi * t)
    return out


def make_affine_sequence(spec: SequenceSpec, dtype=np.float32, smooth: bool = False, gain=None, offset=None,
                         **motion) -> np.ndarray:
    """Frames R_k(x) = gain_k B(x + v_k(x)) + offset_k + N(0, noise_sd^2)
    under affine_motion; B the OCT-like image, or blob_image when smooth;
    gain and offset per frame (default 1 and 0)."""
    speckle = _make_speckle(spec)
    M, s = affine_motion(spec, **motion)
    x = cell_centres(spec.shape)
    d = spec.dim
    c = (np.asarray(spec.shape, dtype=np.float64) / 2.0).reshape((d,) + (1,) * d)
    noise = philox(spec.seed, 3)
    out = np.empty((spec.n,) + tuple(spec.shape), dtype=dtype)
    for k in range(spec.n):
        v = np.tensordot(M[k] - np.eye(d), x - c, axes=(1, 0)) + s[k].reshape((d,) + (1,) * d)
        img = blob_image(spec, x + v) if smooth else base_image(spec, x + v, speckle)
        if gain is not None:
            img = img * float(gain[k])
        if offset is not None:
            img = img + float(offset[k])
        img += noise.normal(scale=spec.noise_sd, size=img.shape) if spec.noise_sd > 0 else 0.0
        out[k] = img.astype(dtype)
    return out
