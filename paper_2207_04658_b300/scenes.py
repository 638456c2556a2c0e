"""Seeded synthetic scenes: initial particle states and the workload definitions.

This module holds no arithmetic of the method (no transfer, no codec, no solve); it only
draws initial positions and states.  Both the CUDA path and the CPU oracle consume what
it produces.  Every draw comes from one Philox stream per scene (numpy's Philox bit
generator keyed by the scene seed).

State layout: float64 array [N, n_comp] in the canonical component order
x[d], v[d], C[d*d] (row major), then F[d*d] (row major) or J for the fluid.

The workloads stand in for the paper's procedural scenes (falling elastic blocks,
Sec. 8.1; dam breaks, Sec. 8.1 and 8.3), at the sizes of the benchmark configurations.
"""
import math

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.Philox(key=int(seed)))


def n_comp(dim, material):
    return 2 * dim + dim * dim + (1 if material == "fluid" else dim * dim)


def jitter_box(gen, lo, size, strata):
    """One uniform sample per stratum of a regular lattice of ``strata`` cells covering
    the axis-aligned box [lo, lo + size).  Returns [prod(strata), d] float64."""
    lo = np.asarray(lo, dtype=np.float64)
    size = np.asarray(size, dtype=np.float64)
    strata = [int(s) for s in strata]
    d = len(strata)
    axes = [np.arange(s, dtype=np.float64) for s in strata]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, d)
    cell = size / np.asarray(strata, dtype=np.float64)
    u = gen.random(grid.shape)
    return lo + (grid + u) * cell


def initial_state(dim, material, x, v0=None):
    """Rest state: given positions, uniform velocity v0, C = 0, F = I (or J = 1)."""
    N = x.shape[0]
    s = np.zeros((N, n_comp(dim, material)), dtype=np.float64)
    s[:, :dim] = x
    if v0 is not None:
        s[:, dim:2 * dim] = np.asarray(v0, dtype=np.float64)
    off = 2 * dim + dim * dim
    if material == "fluid":
        s[:, off] = 1.0
    else:
        for a in range(dim):
            s[:, off + a * dim + a] = 1.0
    return s


def place_cubes(gen, count, side, lo=0.1, hi=0.9, max_tries=100000):
    """Non-overlapping axis-aligned cube corners inside [lo, hi]^3 by rejection."""
    corners = []
    tries = 0
    while len(corners) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place non-overlapping cubes")
        c = lo + gen.random(3) * (hi - lo - side)
        if all(np.any(np.abs(c - o) >= side) for o in corners):
            corners.append(c)
    return np.array(corners)


# ---------------------------------------------------------------------------- workloads
def block2d_scene(n_strata=(128, 64), grid_log2=7, seed=1, steps=500, resort_every=8):
    """2D neo-Hookean block: jitter-sampled in the square [0.4, 0.6]^2 (8,192 particles
    with the default 128 x 64 strata), 128^2 grid, E = 1e3, nu = 0.2, rho = 1,
    g = -9.8, dt = 1e-4, sticky walls."""
    N = int(np.prod(n_strata))
    scene = dict(name="block2d", dim=2, material="neohookean", grid_log2=grid_log2, bound=3,
                 dt=1e-4, E=1e3, nu=0.2, bulk=0.0, rho=1.0, p_vol=0.2 * 0.2 / N,
                 gravity=(0.0, -9.8, 0.0), seed=seed, dither=True, steps=steps,
                 resort_every=resort_every)
    x = jitter_box(rng(seed), (0.4, 0.4), (0.2, 0.2), n_strata)
    return scene, initial_state(2, "neohookean", x)


def block2d_scheme():
    """Fixed 16-bit scheme of the 2D block: x on [0,1) (Delta 2^-16), v on [-4,4]
    (2^-13), C on [-64,64] (2^-9), F on [0,2] (2^-15); bit pack."""
    return {
        "x": dict(bits=16, frac=16, offset=0, container=0),
        "v": dict(bits=16, frac=13, offset=-4 * 2 ** 13, container=0),
        "C": dict(bits=16, frac=9, offset=-64 * 2 ** 9, container=0),
        "F": dict(bits=16, frac=15, offset=0, container=0),
    }


def cubes3d_scene(n_cubes=16, cube_cells=40, ppc_axis=2, grid_log2=8, seed=2, steps=1000,
                  material="corotated", E=5e3, nu=0.3, rho=4.0, dt=5e-5, speed=3.0,
                  resort_every=8):
    """3D elastic cubes (fixed-corotated by default) thrown together: ``n_cubes`` cubes of
    side cube_cells * dx at seeded non-overlapping corners in [0.1, 0.9]^3, ppc_axis^3
    jittered particles per cell (8 by default), each cube moving at ``speed`` toward the
    centre of the domain (plus gravity), so that cubes collide within the run.  The
    defaults give 16 x 512,000 = 8,192,000 particles on a 256^3 grid; with E = 5e3,
    nu = 0.3 and rho = 4 the P-wave speed is 41 m/s and dt = 5e-5 is half the cell
    crossing time (CFL 0.5).  The same seed at half resolution (cube_cells=20,
    grid_log2=7) is the same scene with 1,024,000 particles."""
    n = 1 << grid_log2
    side = cube_cells / n
    gen = rng(seed)
    corners = place_cubes(gen, n_cubes, side)
    strata = (cube_cells * ppc_axis,) * 3
    xs = [jitter_box(gen, c, (side,) * 3, strata) for c in corners]
    x = np.concatenate(xs, axis=0)
    N = x.shape[0]
    per = strata[0] ** 3
    v = np.zeros((N, 3))
    for i, c in enumerate(corners):
        to_centre = 0.5 - (c + 0.5 * side)
        nrm = np.linalg.norm(to_centre)
        if nrm > 0 and speed > 0:
            v[i * per:(i + 1) * per] = speed * to_centre / nrm
    scene = dict(name="cubes3d", dim=3, material=material, grid_log2=grid_log2, bound=3,
                 dt=dt, E=E, nu=nu, bulk=0.0, rho=rho, p_vol=n_cubes * side ** 3 / N,
                 gravity=(0.0, -9.8, 0.0), seed=seed, dither=True, steps=steps,
                 resort_every=resort_every)
    s = initial_state(3, material, x)
    s[:, 3:6] = v
    return scene, s


def dambreak3d_scene(column_cells=256, ppc_axis=2, grid_log2=9, seed=3, steps=500,
                     bulk=400.0, dt=2e-5, resort_every=8):
    """3D weakly compressible dam break: a cubic column of column_cells^3 cells at the
    low corner (starting at the sticky wall, 3 dx), ppc_axis^3 jittered particles per
    cell.  Defaults: 256^3 cells x 8 = 2^27 particles on a 512^3 grid, K = 400."""
    n = 1 << grid_log2
    lo = 3.0 / n
    side = column_cells / n
    x = jitter_box(rng(seed), (lo, lo, lo), (side,) * 3, (column_cells * ppc_axis,) * 3)
    N = x.shape[0]
    scene = dict(name="dambreak3d", dim=3, material="fluid", grid_log2=grid_log2, bound=3,
                 dt=dt, E=0.0, nu=0.0, bulk=bulk, rho=1.0, p_vol=side ** 3 / N,
                 gravity=(0.0, -9.8, 0.0), seed=seed, dither=True, steps=steps,
                 resort_every=resort_every)
    return scene, initial_state(3, "fluid", x)


def fixed_scheme_3d(material, x_bits=21, v=(16, -8.0, 8.0), C=(16, -512.0, 512.0),
                    F=(16, -0.5, 1.5), J=(16, 0.0, 2.0), x_container=64):
    """A hand-written 3D scheme: x as 3 x ``x_bits`` on [0, 1) in one 64-bit container,
    the other fields bit-packed with the given (bits, lo, hi) and the coarsest
    power-of-two resolution whose window covers [lo, hi]."""
    def field(bits, lo, hi):
        k = int(math.floor(bits - math.log2(hi - lo)))
        return dict(bits=bits, frac=k, offset=int(math.floor(lo * 2 ** k)), container=0)
    sch = {"x": dict(bits=x_bits, frac=x_bits, offset=0, container=x_container),
           "v": field(*v), "C": field(*C)}
    if material == "fluid":
        sch["J"] = field(*J)
    else:
        sch["F"] = field(*F)
    return sch


# ---------------------------------------------------------------------------- serving
SERVING_CLASSES = [(2, "neohookean"), (2, "fluid"), (3, "corotated"), (3, "fluid")]
SERVING_GRIDS = {2: (7, 8, 9, 10), 3: (6, 7, 8)}
SERVING_EPS = (0.1, 0.01)
SERVING_STEPS = 200


def _wave_speed(dim, material, E, nu, rho, bulk):
    if material == "fluid":
        return math.sqrt(bulk / rho)
    return math.sqrt(E * (1 - nu) / ((1 + nu) * (1 - 2 * nu)) / rho)


def serving_scene(dim, material, n_particles, grid_log2, seed, steps=SERVING_STEPS):
    """One serving request's scene: an elastic body (2D neo-Hookean E 1e3, nu 0.2, rho 1;
    3D fixed-corotated E 5e3, nu 0.3, rho 4) thrown downward at 1 m/s from the middle of
    the domain, or a fluid column (K 400, rho 1) at the low corner (a dam break).  About
    n_particles jittered particles (k^d strata, k = round(n^(1/d))) in a box of n / ppc
    cells, ppc = 4 (2D) or 8 (3D), capped at 60 % of the domain per axis (denser then);
    dt = 0.3 dx / (wave speed + 1 m/s), at most 1e-4."""
    n = 1 << grid_log2
    dx = 1.0 / n
    ppc = 4 if dim == 2 else 8
    k = max(2, int(round(n_particles ** (1.0 / dim))))
    side_cells = min(0.6 * n, (k ** dim / ppc) ** (1.0 / dim))
    side = side_cells * dx
    gen = rng(seed)
    fluid = material == "fluid"
    if fluid:
        lo = np.full(dim, 3.0 * dx)
    else:
        lo = np.full(dim, 0.5 - side / 2)
        lo[1] = min(0.55, 1.0 - 8 * dx - side)  # the top stays clear of the wall band
    x = jitter_box(gen, lo, np.full(dim, side), (k,) * dim)
    E, nu, rho, bulk = (0.0, 0.0, 1.0, 400.0) if fluid else ((1e3, 0.2, 1.0, 0.0) if dim == 2 else (5e3, 0.3, 4.0, 0.0))
    c = _wave_speed(dim, material, E, nu, rho, bulk)
    dt = min(1e-4, 0.3 * dx / (c + 1.0))
    s0 = initial_state(dim, material, x)
    if not fluid:
        s0[:, dim + 1] = -1.0
    scene = dict(name=f"serve{dim}d_{material}", dim=dim, material=material, grid_log2=grid_log2, bound=3,
                 dt=dt, E=E, nu=nu, bulk=bulk, rho=rho, p_vol=side ** dim / x.shape[0],
                 gravity=(0.0, -9.8, 0.0), seed=seed, dither=True, steps=steps, resort_every=8)
    return scene, s0


def serving_requests(rate=20.0, duration=15.0, seed=5, n_min=1e4, n_max=4e6):
    """Poisson arrivals (rate per second over `duration` seconds) of requests: a class
    (2D/3D x elastic/fluid, uniform), a particle count log-uniform in [n_min, n_max], a
    grid uniform over the class's resolutions (raised to the first one whose 60 % box holds
    the particles at no more than 32 per cell), an error bound from {0.1, 0.01} and 200
    steps.  Returns a list of dicts (t, dim, material, n, grid_log2, eps, seed)."""
    gen = rng(seed)
    t = 0.0
    out = []
    while True:
        t += float(gen.exponential(1.0 / rate))
        if t > duration:
            return out
        dim, material = SERVING_CLASSES[int(gen.integers(0, len(SERVING_CLASSES)))]
        n = int(round(math.exp(gen.uniform(math.log(n_min), math.log(n_max)))))
        grids = SERVING_GRIDS[dim]
        gi = int(gen.integers(0, len(grids)))
        while gi + 1 < len(grids) and n > 32 * (0.6 * (1 << grids[gi])) ** dim:
            gi += 1
        eps = SERVING_EPS[int(gen.integers(0, len(SERVING_EPS)))]
        out.append(dict(t=t, dim=dim, material=material, n=n, grid_log2=grids[gi], eps=eps,
                        seed=int(gen.integers(1, 2 ** 31))))


# ------------------------------------------------------------------------------ smoke
def smoke_scene(n=256, jacobi=64, steps=100, seed=7):
    """The 2D smoke plume of the error-bounded experiment (Sec. 8.1: 256^2 grid, dt 0.01,
    RK-3 advection, 64 Jacobi sweeps, z = sum of squared density): a source box at the
    bottom centre (density 1, inflow 1) with buoyancy 1, run for `steps` steps from rest.
    The paper prints neither the source nor the step count; this plume reaches the top of
    the box within the run and gives z of the order of the paper's (about 2e4)."""
    return dict(n=n, jacobi=jacobi, dt=0.01, buoyancy=1.0, v_in=1.0, src=(0.35, 0.05, 0.65, 0.12), seed=seed,
                steps=steps)


# ------------------------------------------------------------------------ memory bound
def dambreak2d_scene(n_particles=10_000, grid_log2=7, steps=16_384, seed=9):
    """The 2D fluid dam break of the memory-bounded experiment (Sec. 8.1: 10,000 particles,
    128^2 grid, 16,384 steps of 2e-4 s, J tracked instead of F, kinetic energy at the final
    step): a jittered column of 100 x 100 strata over [0.05, 0.45]^2 at the low corner,
    K = 100 (wave speed 10 m/s: 0.26 dx per step), rho 1, gravity -9.8.  The paper prints
    neither the column nor K."""
    n = 1 << grid_log2
    k = int(round(n_particles ** 0.5))
    gen = rng(seed)
    x = jitter_box(gen, np.array([0.05, 0.05]), np.array([0.4, 0.4]), (k, k))
    s0 = initial_state(2, "fluid", x)
    scene = dict(name="dambreak2d", dim=2, material="fluid", grid_log2=grid_log2, bound=3, dt=2e-4, E=0.0, nu=0.0,
                 bulk=100.0, rho=1.0, p_vol=0.16 / x.shape[0], gravity=(0.0, -9.8, 0.0), seed=seed, dither=True,
                 steps=steps, resort_every=8)
    return scene, s0


# --------------------------------------------------------------------------- scaling
SCALING_CONFIGS = [  # (particles, grid log2, dt, steps): Sec. 8.3's refinement sequence
    (200_000, 6, 2e-4, 16_384),
    (500_000, 6, 2e-4, 16_384),
    (1_000_000, 7, 1e-4, 32_768),
    (5_000_000, 8, 5e-5, 65_536),
]


def fluid3d_column_scene(n_particles, grid_log2, dt, steps, seed=11):
    """The 3D fluid of the scaling experiment (Sec. 8.3): a column of constant initial
    volume, [0.1, 0.5] x [0.1, 0.6] x [0.1, 0.5], sampled by k^3 jittered strata (k = the
    cube root of the particle count), K = 200, rho 1, gravity -9.8; the evaluation is the
    particles' mean height.  The paper prints neither the column nor K."""
    k = int(round(n_particles ** (1.0 / 3.0)))
    gen = rng(seed)
    lo, size = np.array([0.1, 0.1, 0.1]), np.array([0.4, 0.5, 0.4])
    x = jitter_box(gen, lo, size, (k, k, k))
    s0 = initial_state(3, "fluid", x)
    scene = dict(name=f"fluid3d_{x.shape[0]}", dim=3, material="fluid", grid_log2=grid_log2, bound=3, dt=dt,
                 E=0.0, nu=0.0, bulk=200.0, rho=1.0, p_vol=float(np.prod(size)) / x.shape[0],
                 gravity=(0.0, -9.8, 0.0), seed=seed, dither=True, steps=steps, resort_every=8)
    return scene, s0
