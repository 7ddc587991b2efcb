"""Seeded synthetic workloads shared by the tests, the smoke check and the benchmark.

Parameters only: patch layouts, motion laws, pulse parameters, time steps
and random arrays.  None of the method's arithmetic lives here; both the CUDA
library and the CPU oracle receive these numbers and evaluate everything
themselves.  Seeds are ``numpy.random.default_rng(20020088 + index)`` with a
fixed draw order, so every workload is reproducible bit for bit.

The paper evaluates on no public dataset: its tests use closed-form plane
waves (Sec. 3).  The throughput workloads here follow the same recipe with
Gaussian-pulse closed forms:

* ``static_gauss``   -- global 48^3 on [-1,1]^3 plus one static local 32^3 at
  2x resolution centred on the origin, one Gaussian pulse (A = 1, width 0.1,
  centre uniform in [-0.2,0.2]^3), 5-point Lagrange, CFL 0.25, 100 steps.
* ``plane_gauss``    -- the precision configuration: global 512^3 (periodic)
  plus one static local 256^3 at 2x, plane wave k = (2,3,5) pi plus one
  Gaussian pulse; 200 steps.
* ``orbiting_gauss`` -- global 256^3 on [-1,1]^3 plus four local 128^3 patches
  (half-width 0.25, 2x resolution) on circular orbits of radius 0.4 and
  angular speed 2 pi in the planes z = +-0.3 (pairs opposite in phase, pair
  phases seeded), eight Gaussians (amplitudes N(0,1), widths U[0.05,0.2],
  centres U[-1,1]^3), 6-point Lagrange, CFL 0.25, 200 steps.
* ``spinning_gauss`` -- the rotating-patch configuration: global 256^3 plus
  four local 96^3 cubes (half-width 3/16, 2x resolution) centred at
  (+-0.45, +-0.45, 0), each spinning about its centre around a seeded unit
  axis at angular speed pi (seeded sign and phase); eight Gaussians as in
  ``orbiting_gauss``; 200 steps.
* ``rotating_plane`` -- the rotating local patch of Sec. 3.2 (Test Two) at
  reduced size, for the convergence pin and the small parity cases.
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

SEED_BASE = 20020088

GLOBAL, LOCAL = 0, 1
BC_ANALYTIC, BC_PERIODIC, BC_INTERPATCH = 0, 1, 2
STATIC, LINEAR, CIRCULAR, ROTATING = 0, 1, 2, 3
CARTESIAN, SPHERICAL = 0, 1
GAUSS_SUM, PLANE_SUM, HARMONIC_POLY, PLANE_GAUSS = 0, 1, 2, 3


@dataclass
class PatchSpec:
    kind: int
    n: Tuple[int, int, int]
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    outer_bc: int
    motion: int = STATIC
    motion_params: Tuple[float, ...] = ()
    topology: int = 0  # CARTESIAN, or SPHERICAL for a local shell (numeric r, theta, phi)


@dataclass
class Workload:
    name: str
    patches: List[PatchSpec]
    analytic_kind: int
    analytic_params: np.ndarray
    analytic_count: int
    interp_points: int
    ko_eps: float
    dt: float
    steps: int
    extra: dict = field(default_factory=dict)

    @property
    def interior_points(self):
        return sum(int(np.prod(p.n)) for p in self.patches)


def rng(index):
    return np.random.default_rng(SEED_BASE + index)


def static_gauss(scale=1, steps=100, interp_points=5, seed_index=0):
    """Static global + one local patch; ``scale`` multiplies both resolutions."""
    r = rng(seed_index)
    centre = r.uniform(-0.2, 0.2, 3)
    ng, nl = 48 * scale, 32 * scale
    third = 1.0 / 3.0
    patches = [
        PatchSpec(GLOBAL, (ng, ng, ng), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), BC_ANALYTIC),
        PatchSpec(LOCAL, (nl, nl, nl), (-third, -third, -third), (third, third, third), BC_INTERPATCH),
    ]
    h_min = (2.0 * third) / nl
    params = np.array([1.0, 0.1, centre[0], centre[1], centre[2]])
    return Workload(f"static_gauss_{ng}+{nl}", patches, GAUSS_SUM, params, 1, interp_points, 0.005,
                    0.25 * h_min, steps, {"centre": centre})


def orbiting_gauss(scale=1, steps=200, interp_points=6, seed_index=1, radius=0.4, omega=2.0 * np.pi,
                   plane_z=0.3, half_width=0.25):
    """Global 256^3/scale + four orbiting local 128^3/scale patches."""
    r = rng(seed_index)
    pair_phase = r.uniform(0.0, 2.0 * np.pi, 2)
    amps = r.normal(0.0, 1.0, 8)
    widths = r.uniform(0.05, 0.2, 8)
    centres = r.uniform(-1.0, 1.0, (8, 3))
    ng, nl = 256 // scale, 128 // scale
    patches = [PatchSpec(GLOBAL, (ng, ng, ng), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), BC_ANALYTIC)]
    for pair, z in enumerate((plane_z, -plane_z)):
        for member in range(2):
            phase = pair_phase[pair] + member * np.pi
            patches.append(PatchSpec(LOCAL, (nl, nl, nl), (-half_width,) * 3, (half_width,) * 3, BC_INTERPATCH,
                                     CIRCULAR, (0.0, 0.0, z, radius, omega, phase)))
    params = np.column_stack([amps, widths, centres]).ravel()
    h_min = 2.0 * half_width / nl
    return Workload(f"orbiting_gauss_{ng}+4x{nl}", patches, GAUSS_SUM, params, 8, interp_points, 0.005,
                    0.25 * h_min, steps)


def spinning_gauss(scale=1, steps=200, interp_points=6, seed_index=4, centre=0.45, omega=np.pi,
                   half_width=0.1875):
    """Global 256^3/scale + four local 96^3/scale cubes spinning in place
    (ROTATING motion: centre fixed, seeded unit axis, angular speed +-omega,
    seeded phase).  The rotated cubes keep an L-infinity gap of >= 0.1 between
    their bounding boxes and stay >= 0.05 inside the global box at every
    angle for scale 1 and 2."""
    r = rng(seed_index)
    axes = r.normal(0.0, 1.0, (4, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    signs = np.where(r.uniform(0.0, 1.0, 4) < 0.5, -1.0, 1.0)
    phases = r.uniform(0.0, 2.0 * np.pi, 4)
    amps = r.normal(0.0, 1.0, 8)
    widths = r.uniform(0.05, 0.2, 8)
    centres = r.uniform(-1.0, 1.0, (8, 3))
    ng, nl = 256 // scale, 96 // scale
    patches = [PatchSpec(GLOBAL, (ng, ng, ng), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), BC_ANALYTIC)]
    for q, (cx, cy) in enumerate(((centre, centre), (-centre, centre), (-centre, -centre), (centre, -centre))):
        patches.append(PatchSpec(LOCAL, (nl, nl, nl), (-half_width,) * 3, (half_width,) * 3, BC_INTERPATCH,
                                 ROTATING, (cx, cy, 0.0, 0.0, 0.0, 0.0, axes[q, 0], axes[q, 1], axes[q, 2],
                                            signs[q] * omega, phases[q])))
    params = np.column_stack([amps, widths, centres]).ravel()
    h_min = 2.0 * half_width / nl
    return Workload(f"spinning_gauss_{ng}+4x{nl}", patches, GAUSS_SUM, params, 8, interp_points, 0.005,
                    0.25 * h_min, steps)


def rotating_plane(scale=1, steps=16, interp_points=6, omega=2.0 * np.pi, axis=(0.0, 0.0, 1.0), half_width=0.3,
                   nl=20, phase=0.0, velocity=(0.0, 0.0, 0.0)):
    """Sec. 3.2's rotating local patch (Test Two) at reduced size: global
    cube [-1,1]^3 at 32 scale cells per axis and a local cube of the given
    half-width (nl scale cells) whose centre sits at the global origin (or
    moves with the given velocity) and which turns counter-clockwise about
    the unit axis at angular speed omega; the two-wave superposition of
    ``translating_plane`` with analytic outer BCs."""
    ng, nl = 32 * scale, nl * scale
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    patches = [
        PatchSpec(GLOBAL, (ng, ng, ng), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), BC_ANALYTIC),
        PatchSpec(LOCAL, (nl, nl, nl), (-half_width,) * 3, (half_width,) * 3, BC_INTERPATCH, ROTATING,
                  (0.0, 0.0, 0.0) + tuple(velocity) + tuple(ax) + (omega, phase)),
    ]
    k = 2.0 * np.pi / 2.0
    params = np.array([3.0, 1.0, k, 0.0, 0.0, 0.0, 1.0, k, -k, k, 0.5 * np.pi])
    h_min = 2.0 * half_width / nl
    return Workload(f"rotating_plane_{ng}+{nl}", patches, PLANE_SUM, params, 2, interp_points, 0.005,
                    0.25 * h_min, steps * scale)


def shell_plane(scale=1, steps=16, interp_points=6, r=(0.3, 0.7), theta=(np.pi / 4, 3 * np.pi / 4), n=(12, 24, 96),
                centre=(0.013, -0.021, 0.017), motion=STATIC, motion_params=None):
    """A spherical local shell (the paper's spherical local patch, Sec. 3.3:
    theta in [pi/4, 3 pi/4], full azimuth) inside the global cube [-1,1]^3 at
    32 scale cells per axis, static at `centre` unless a motion law is
    given; n = (r, theta, phi) cells at scale 1.  The two-wave superposition
    of ``translating_plane`` with analytic outer BCs; dt = CFL 0.25 times the
    smallest physical spacing of the shell (the azimuthal one at r_lo,
    theta_lo)."""
    ng = 32 * scale
    ns = tuple(int(v) * scale for v in n)
    mp = tuple(centre) if motion_params is None else tuple(motion_params)
    patches = [
        PatchSpec(GLOBAL, (ng, ng, ng), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), BC_ANALYTIC),
        PatchSpec(LOCAL, ns, (r[0], theta[0], 0.0), (r[1], theta[1], 2.0 * np.pi), BC_INTERPATCH, motion, mp,
                  SPHERICAL),
    ]
    k = 2.0 * np.pi / 2.0
    params = np.array([3.0, 1.0, k, 0.0, 0.0, 0.0, 1.0, k, -k, k, 0.5 * np.pi])
    h = [(r[1] - r[0]) / ns[0], r[0] * (theta[1] - theta[0]) / ns[1],
         r[0] * np.sin(theta[0]) * 2.0 * np.pi / ns[2]]
    return Workload(f"shell_plane_{ng}+{ns[0]}x{ns[1]}x{ns[2]}", patches, PLANE_SUM, params, 2, interp_points, 0.005,
                    0.25 * min(h), steps * scale)


def plane_gauss(scale=1, steps=200, interp_points=6, seed_index=2):
    """The precision configuration: the static layout of ``static_gauss`` at global
    512^3/scale on the periodic box [-1,1]^3 and one local 256^3/scale patch of
    half-width 0.25 (2x resolution) centred on the origin.  Initial data: the
    plane wave k = (2, 3, 5) pi (period 2 on every axis, so the periodic box
    holds it exactly; amplitude 1, phase seeded) plus one Gaussian pulse
    (A = 1, width 0.1, centre uniform in [-0.2,0.2]^3), whose tail at the box
    faces is below 1e-40 and which travels 0.1 in 200 steps.  CFL 0.25 on the
    local spacing."""
    r = rng(seed_index)
    phase = r.uniform(0.0, 2.0 * np.pi)
    centre = r.uniform(-0.2, 0.2, 3)
    ng, nl = 512 // scale, 256 // scale
    patches = [
        PatchSpec(GLOBAL, (ng, ng, ng), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), BC_PERIODIC),
        PatchSpec(LOCAL, (nl, nl, nl), (-0.25, -0.25, -0.25), (0.25, 0.25, 0.25), BC_INTERPATCH),
    ]
    k = np.pi * np.array([2.0, 3.0, 5.0])
    params = np.array([0.0, 1.0, k[0], k[1], k[2], phase, 1.0, 0.1, centre[0], centre[1], centre[2]])
    h_min = 0.5 / nl
    return Workload(f"plane_gauss_{ng}+{nl}", patches, PLANE_GAUSS, params, 1, interp_points, 0.005,
                    0.25 * h_min, steps, {"centre": centre, "phase": phase})


def shell_instance(ng, rs, moving):
    """One spherical shell r in [0.1, 0.5], theta in [pi/4, 3 pi/4], full
    azimuth, for a global n_g^3 on [-1,1]^3: physical spacings at most the
    global one (n_r, n_theta, n_phi rounded up to multiples of 4, 4, 8), centre
    U[-0.05,0.05]^3, spinning about its local z axis at a seeded angular speed
    up to pi when moving."""
    hg = 2.0 / ng
    up = lambda x, m: int(np.ceil(x / m) * m)
    n = (up(0.4 / hg, 4), up(0.5 * (np.pi / 2) / hg, 4), up(0.5 * 2 * np.pi / hg, 8))
    c = rs.uniform(-0.05, 0.05, 3)
    omega, phase = rs.uniform(-np.pi, np.pi), rs.uniform(0.0, 2.0 * np.pi)
    mp = (tuple(c) + (0.0, 0.0, 0.0, 0.0, 0.0, 1.0, omega, phase)) if moving else tuple(c)
    spec = PatchSpec(LOCAL, n, (0.1, np.pi / 4, 0.0), (0.5, 3 * np.pi / 4, 2 * np.pi), BC_INTERPATCH,
                     ROTATING if moving else STATIC, mp, SPHERICAL)
    dmin = min(0.4 / n[0], 0.1 * (np.pi / 2) / n[1], 0.1 * np.sin(np.pi / 4) * 2 * np.pi / n[2])
    return spec, 0.25 * dmin


def batch_instances(count=64, steps=100, seed_index=3, interp_points=6, max_global=192, moving=True, shells=False):
    """Independent instances of uneven sizes for a batched run.

    Instance k: a global cube of n_g^3 (n_g from 64 to ``max_global`` in steps
    of 32) on [-1,1]^3 with the analytic outer BC, and 1 to 8 local cubes of
    n_l^3 at 2x resolution (n_l from 32 to n_g/2), one per octant of the
    global box, each centred in its octant and moving with a seeded constant
    velocity of at most 0.5.  The velocity is capped so that after ``steps``
    steps of dt = h_local/4 the cube keeps its containment margin and its
    gap to the neighbouring octants.  Initial data: two Gaussian pulses
    (amplitudes N(0,1), widths U[0.08,0.2], centres U[-0.8,0.8]^3).  With
    ``moving=False`` every local cube stays at its octant centre.  With
    ``shells=True`` every second instance holds one spherical shell
    (``shell_instance``, drawn from a second seeded generator) in place of its
    local cubes."""
    r = rng(seed_index)
    rs = rng(50 + seed_index)
    out = []
    sizes = [n for n in range(64, max_global + 1, 32)]
    for k in range(count):
        ng = int(r.choice(sizes))
        nloc = int(r.integers(1, 9))
        nl = int(r.choice([n for n in range(32, ng // 2 + 1, 16)]))
        h0, hl = 2.0 / ng, 1.0 / ng
        dt = 0.25 * hl
        ext = nl * hl                       # local cube edge
        margin = 3 * hl + 8 * h0            # to the octant walls (containment, gaps)
        room = 0.5 * (1.0 - ext) - margin   # free travel inside the octant
        vmax = max(0.0, min(0.5, room / (steps * dt))) if moving else 0.0
        octs = r.permutation(8)[:nloc]
        patches = [PatchSpec(GLOBAL, (ng, ng, ng), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), BC_ANALYTIC)]
        for o in octs:
            c = np.array([0.5 if (o >> a) & 1 else -0.5 for a in range(3)])
            d = r.normal(size=3)
            v = d / np.linalg.norm(d) * r.uniform(0.0, vmax)
            half = 0.5 * ext
            patches.append(PatchSpec(LOCAL, (nl, nl, nl), (-half,) * 3, (half,) * 3, BC_INTERPATCH, LINEAR,
                                     (c[0], c[1], c[2], v[0], v[1], v[2])))
        params = np.column_stack([r.normal(0.0, 1.0, 2), r.uniform(0.08, 0.2, 2),
                                  r.uniform(-0.8, 0.8, (2, 3))]).ravel()
        name = f"instance{k}_{ng}+{nloc}x{nl}"
        if shells and k % 2 == 1:
            spec, dt = shell_instance(ng, rs, moving)
            patches = patches[:1] + [spec]
            name = f"instance{k}_{ng}+shell{spec.n[0]}x{spec.n[1]}x{spec.n[2]}"
        out.append(Workload(name, patches, GAUSS_SUM, params, 2, interp_points, 0.005, dt, steps))
    return out


def translating_plane(scale=1, steps=16, interp_points=6, velocity=(0.4, 0.3, 0.0), start=(-0.05, -0.02, 0.0)):
    """Sec. 3.2-style convergence layout at reduced size: global cube [-1,1]^3
    and a 2:1 local cube [-0.5,0.5]^3 translating with constant velocity,
    evolving the two-wave superposition of Sec. 3.4.2 scaled to the box
    (wavelengths L1 = L2 = 2, offset 3)."""
    ng, nl = 32 * scale, 32 * scale
    patches = [
        PatchSpec(GLOBAL, (ng, ng, ng), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), BC_ANALYTIC),
        PatchSpec(LOCAL, (nl, nl, nl), (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), BC_INTERPATCH, LINEAR,
                  tuple(start) + tuple(velocity)),
    ]
    k = 2.0 * np.pi / 2.0
    params = np.array([3.0, 1.0, k, 0.0, 0.0, 0.0, 1.0, k, -k, k, 0.5 * np.pi])
    h_min = 1.0 / nl
    return Workload(f"translating_plane_{ng}+{nl}", patches, PLANE_SUM, params, 2, interp_points, 0.005,
                    0.25 * h_min, steps * scale)


def random_fields(shape, seed_index, scale=1.0):
    """Two independent standard-normal arrays of the given shape."""
    r = rng(100 + seed_index)
    return scale * r.standard_normal(shape), scale * r.standard_normal(shape)


def random_offsets(count, seed_index, low, high):
    return rng(200 + seed_index).uniform(low, high, (count, 3))


# ---------------------------------------------------------------- learned surrogate inputs

def surrogate_pulses(seed_index, count=8, spread=0.5):
    """GAUSS_SUM parameters of one training or test state: `count` Gaussians,
    amplitudes N(0,1), widths U[0.05,0.2], centres U[-spread,spread]^3 (on the
    periodic box [-1,1]^3 the widest pulse is below 2e-3 at the faces)."""
    r = rng(seed_index)
    amps = r.normal(0.0, 1.0, count)
    widths = r.uniform(0.05, 0.2, count)
    centres = r.uniform(-spread, spread, (count, 3))
    return np.column_stack([amps, widths, centres]).ravel()


# (cin, cout, relu) of the four layers and their stored channel counts
SURROGATE_LAYERS = [(7, 32, True), (32, 32, True), (32, 32, True), (32, 2, False)]
SURROGATE_PADDED = [(8, 32), (32, 32), (32, 32), (32, 8)]


def surrogate_init(seed_index):
    """Initial parameters in the flat padded binary32 layout of
    include/mpw_surrogate.h: He-scaled normal weights for the ReLU layers, a
    last layer at 0.1 of that scale, zero biases and zero padding."""
    r = rng(seed_index)
    parts = []
    for (ci, co, relu), (pci, pco) in zip(SURROGATE_LAYERS, SURROGATE_PADDED):
        std = np.sqrt(2.0 / (27 * ci)) if relu else 0.1 / np.sqrt(27 * ci)
        W = np.zeros((pco, 27, pci))
        W[:co, :, :ci] = r.standard_normal((co, 27, ci)) * std
        parts += [W.ravel(), np.zeros(pco)]
    return np.concatenate(parts).astype(np.float32)


def surrogate_layout(scale=1, steps=400, seed_index=7, interp_points=6):
    """The learned-surrogate configuration: a periodic global 128^3/scale on
    [-1,1]^3 (advanced four steps per network call) and two local 64^3/scale
    patches at 2x resolution (half-width 0.25) on circular orbits of radius
    0.4, angular speed 2 pi, in the planes z = +0.3 and z = -0.3 (phases
    seeded), which stay on the plain method; eight Gaussians as in
    ``surrogate_pulses``; CFL 0.25 on the local spacing; 400 steps."""
    r = rng(seed_index)
    phases = r.uniform(0.0, 2.0 * np.pi, 2)
    ng, nl = 128 // scale, 64 // scale
    patches = [PatchSpec(GLOBAL, (ng, ng, ng), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), BC_PERIODIC)]
    for z, ph in zip((0.3, -0.3), phases):
        patches.append(PatchSpec(LOCAL, (nl, nl, nl), (-0.25,) * 3, (0.25,) * 3, BC_INTERPATCH, CIRCULAR,
                                 (0.0, 0.0, z, 0.4, 2.0 * np.pi, ph)))
    params = surrogate_pulses(seed_index + 1)
    h_min = 0.5 / nl
    return Workload(f"surrogate_{ng}+2x{nl}", patches, GAUSS_SUM, params, 8, interp_points, 0.005, 0.25 * h_min,
                    steps)
