"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs (positions, vacant-element counts, signal types,
spike flags, retraction counts). It holds none of the method's arithmetic, so
both the CUDA path and the CPU oracle consume exactly the same arrays.

The paper (Sec. V-B) simulates networks from empty connectivity with 1.1-1.5
vacant elements per neuron and states no spatial distribution; the layouts
below stand in for it:

* ``uniform_cube``   - uniform positions in a cube, U{0..4} vacancies (4096 neurons
  in a 1000 um cube is the small parity case).
* ``gaussian_clusters`` - 64 isotropic Gaussian clusters (std 300 um) with centres
  uniform in a 10 mm cube, Poisson(2) vacancies clipped to 0..8 (2^20 neurons,
  2^14 per cluster, is the headline benchmark workload).
* ``cortical_slab``  - 20 x 20 x 2.5 mm slab of 10 layers, uniform within a layer,
  layer shares 1 + U(-0.3, 0.3) normalised, Poisson(1) vacancies (2^24 neurons).
* ``differentiable_cube`` - uniform positions in a cube, Poisson(2) vacancies
  clipped to 0..8, sigma 800 um (2^18 neurons in a 4 mm cube is the
  differentiable form's workload; smaller n keeps the density by default).
* ``network_batch``  - many independent networks of uneven sizes (log-uniform
  neuron counts), each uniform in its own cube at the density of ``uniform_cube``
  (4096 neurons per mm^3), Poisson(2) vacancies clipped to 0..8, per-network sigma
  uniform in [500, 1000] um (256 networks of 10^3 .. 10^6 neurons, about 3.7e7 in
  total, is the batched workload).

Every generator is keyed by an integer seed through NumPy's Philox bit
generator; 20 % of neurons are inhibitory (type 1), drawn i.i.d.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Network:
    name: str
    x: np.ndarray          # float32 [n], micrometres
    y: np.ndarray
    z: np.ndarray
    vac_ax: np.ndarray     # int32 [n] vacant axonal elements
    vac_de: np.ndarray     # int32 [n] vacant dendritic elements
    type: np.ndarray       # uint8 [n] 0 = excitatory, 1 = inhibitory
    sigma: float           # kernel width, micrometres
    theta: float           # Barnes-Hut acceptance parameter
    seed: int              # key of the method's Philox draws
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, stream]))


def _types(rng, n, p_inh=0.2):
    return (rng.random(n) < p_inh).astype(np.uint8)


def _poisson(rng, lam, n, hi=8):
    return np.clip(rng.poisson(lam, n), 0, hi).astype(np.int32)


def uniform_cube(n=4096, side=1000.0, seed=1, sigma=750.0, theta=0.3, vac_max=4):
    """Positions uniform in [0, side]^3, vacancies uniform in {0..vac_max}."""
    rng = _rng(seed)
    p = (rng.random((3, n)) * side).astype(np.float32)
    vac_ax = rng.integers(0, vac_max + 1, n).astype(np.int32)
    vac_de = rng.integers(0, vac_max + 1, n).astype(np.int32)
    return Network("uniform_cube", p[0].copy(), p[1].copy(), p[2].copy(), vac_ax, vac_de,
                   _types(rng, n), float(sigma), float(theta), int(seed),
                   {"n": n, "side_um": side, "vacancies": f"U{{0..{vac_max}}}"})


def differentiable_cube(n=1 << 18, side=None, seed=5, sigma=800.0, theta=0.3, lam=2.0):
    """Positions uniform in [0, side]^3; side defaults to 4 mm at 2^18 neurons and keeps
    that density at other n (1 mm at 2^12)."""
    if side is None:
        side = 4000.0 * (n / float(1 << 18)) ** (1.0 / 3.0)
    rng = _rng(seed)
    p = (rng.random((3, n)) * side).astype(np.float32)
    return Network("differentiable_cube", p[0].copy(), p[1].copy(), p[2].copy(),
                   _poisson(rng, lam, n), _poisson(rng, lam, n), _types(rng, n), float(sigma),
                   float(theta), int(seed),
                   {"n": n, "side_um": side, "vacancies": f"Poisson({lam}) clipped 0..8"})


def gaussian_clusters(n=1 << 20, clusters=64, side=10000.0, std=300.0, seed=2, sigma=750.0,
                      theta=0.3, lam=2.0):
    """``clusters`` isotropic Gaussian clusters of equal size (the remainder goes
    to the first clusters), centres uniform in [0, side]^3."""
    rng = _rng(seed)
    centres = rng.random((clusters, 3)) * side
    sizes = np.full(clusters, n // clusters, np.int64)
    sizes[: n - int(sizes.sum())] += 1
    owner = np.repeat(np.arange(clusters), sizes)
    p = centres[owner] + rng.normal(0.0, std, (n, 3))
    p = p.astype(np.float32)
    return Network("gaussian_clusters", p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(),
                   _poisson(rng, lam, n), _poisson(rng, lam, n), _types(rng, n), float(sigma),
                   float(theta), int(seed),
                   {"n": n, "clusters": clusters, "side_um": side, "std_um": std,
                    "vacancies": f"Poisson({lam}) clipped 0..8"})


def cortical_slab(n=1 << 24, sx=20000.0, sy=20000.0, sz=2500.0, layers=10, seed=3,
                  sigma=1000.0, theta=0.3, lam=1.0):
    """Layered slab: layer shares 1 + U(-0.3, 0.3), normalised; uniform in a layer."""
    rng = _rng(seed)
    share = 1.0 + rng.uniform(-0.3, 0.3, layers)
    share /= share.sum()
    sizes = np.floor(share * n).astype(np.int64)
    sizes[: n - int(sizes.sum())] += 1
    layer = np.repeat(np.arange(layers), sizes)
    x = (rng.random(n) * sx).astype(np.float32)
    y = (rng.random(n) * sy).astype(np.float32)
    z = ((layer + rng.random(n)) * (sz / layers)).astype(np.float32)
    return Network("cortical_slab", x, y, z, _poisson(rng, lam, n), _poisson(rng, lam, n),
                   _types(rng, n), float(sigma), float(theta), int(seed),
                   {"n": n, "slab_um": [sx, sy, sz], "layers": layers,
                    "vacancies": f"Poisson({lam})"})


def spikes(n, seed, step, p=0.05):
    """Spike flags for one simulation step, i.i.d. Bernoulli(p)."""
    rng = _rng(seed, 1000 + int(step))
    return (rng.random(n) < p).astype(np.uint8)


def retractions(n, seed, step, lam=0.5):
    """Retraction counts for one deletion pass (axonal, dendritic), Poisson(lam)."""
    rng = _rng(seed, 5000 + int(step))
    return (np.minimum(rng.poisson(lam, n), 8).astype(np.int32),
            np.minimum(rng.poisson(lam, n), 8).astype(np.int32))


def regrowth(n, seed, step, lam=1.0):
    """Vacant elements added by the (out-of-scope) element model between updates."""
    rng = _rng(seed, 9000 + int(step))
    return (np.minimum(rng.poisson(lam, n), 8).astype(np.int32),
            np.minimum(rng.poisson(lam, n), 8).astype(np.int32))


@dataclass
class NetworkBatch:
    """Independent networks packed into one id range: network b holds the ids
    offsets[b] .. offsets[b + 1] - 1."""
    name: str
    offsets: np.ndarray    # int64 [B + 1]
    x: np.ndarray          # float32 [n], each network in its own frame
    y: np.ndarray
    z: np.ndarray
    vac_ax: np.ndarray
    vac_de: np.ndarray
    type: np.ndarray
    sigma: np.ndarray      # float32 [B], per-network kernel width
    theta: float
    seed: int
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.offsets[-1])

    @property
    def num_networks(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def network(self, b: int) -> Network:
        lo, hi = int(self.offsets[b]), int(self.offsets[b + 1])
        return Network(f"{self.name}[{b}]", self.x[lo:hi], self.y[lo:hi], self.z[lo:hi],
                       self.vac_ax[lo:hi], self.vac_de[lo:hi], self.type[lo:hi],
                       float(self.sigma[b]), self.theta, self.seed, {"id_base": lo})


def network_batch(networks=256, n_min=1000, n_max=1000000, seed=4, density_per_mm3=4096.0,
                  sigma_lo=500.0, sigma_hi=1000.0, theta=0.3, lam=2.0, sizes=None):
    """``networks`` independent networks, neuron counts log-uniform in [n_min, n_max]
    (or the given ``sizes``), each uniform in [0, side_b]^3 with side_b chosen for a
    constant density, sigma_b ~ U[sigma_lo, sigma_hi]."""
    rng = _rng(seed)
    if sizes is None:
        sizes = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), networks)))
    sizes = np.asarray(sizes, np.int64)
    assert sizes.min() >= 1
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offsets[-1])
    side = (sizes / density_per_mm3) ** (1.0 / 3.0) * 1000.0  # micrometres
    owner = np.repeat(np.arange(sizes.shape[0]), sizes)
    p = (rng.random((3, n)) * side[owner]).astype(np.float32)
    sigma = rng.uniform(sigma_lo, sigma_hi, sizes.shape[0]).astype(np.float32)
    return NetworkBatch("network_batch", offsets, p[0].copy(), p[1].copy(), p[2].copy(),
                        _poisson(rng, lam, n), _poisson(rng, lam, n), _types(rng, n), sigma,
                        float(theta), int(seed),
                        {"networks": int(sizes.shape[0]), "n": n,
                         "sizes": "log-uniform" if n_min != n_max else "equal",
                         "n_range": [int(sizes.min()), int(sizes.max())],
                         "density_per_mm3": density_per_mm3,
                         "sigma_um": [sigma_lo, sigma_hi],
                         "vacancies": f"Poisson({lam}) clipped 0..8"})
