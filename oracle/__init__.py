"""CPU oracle for the quantized MLS-MPM step (ctypes wrapper over ``liboracle.so``).

TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded FP64 C that restates what the
hot path computes, written from the paper ("Automatic Quantization for Physics-Based
Simulation", Liu et al. 2022): the fixed-point codec of Sec. 3.1 (Eq. 3), the dithered
store of Sec. 5 (Eq. 11), the bit pack placement of Sec. 7, the quantized step of
Eq. 1 on the MLS-MPM simulator of Sec. 8.1 and the bit-allocation solve of Sec. 4
(Eq. 6-10, Algorithm 1).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import it.  It shares no code with
the CUDA library and never imports it.
"""
import ctypes as ct
import os

import numpy as np

from . import build as _build

_lib = None
_lib_omp = None

NEOHOOKEAN, COROTATED, FLUID = 0, 1, 2
MATERIALS = {"neohookean": NEOHOOKEAN, "corotated": COROTATED, "fluid": FLUID}
MAX_COMP = 24
N_STATS = 13


class Phys(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("material", ct.c_int), ("grid_log2", ct.c_int),
                ("bound", ct.c_int), ("dt", ct.c_double), ("E", ct.c_double),
                ("nu", ct.c_double), ("bulk", ct.c_double), ("p_vol", ct.c_double),
                ("p_mass", ct.c_double), ("gravity", ct.c_double * 3)]


class Codec(ct.Structure):
    _fields_ = [("n_comp", ct.c_int), ("n_words", ct.c_int),
                ("bits", ct.c_int * MAX_COMP), ("frac", ct.c_int * MAX_COMP),
                ("offset", ct.c_int64 * MAX_COMP), ("bitpos", ct.c_int * MAX_COMP),
                ("field", ct.c_int * MAX_COMP), ("seed", ct.c_uint64), ("dither", ct.c_int)]


class SolveIn(ct.Structure):
    _fields_ = [("H", ct.c_int), ("P", ct.c_double * 8), ("g", ct.c_double * 8),
                ("lo", ct.c_double * 8), ("hi", ct.c_double * 8), ("kappa", ct.c_double),
                ("z", ct.c_double), ("eps", ct.c_double), ("mode", ct.c_int),
                ("rounding", ct.c_int)]


class SolveOut(ct.Structure):
    _fields_ = [("delta_cont", ct.c_double * 8), ("bits_paper", ct.c_int * 8),
                ("bits", ct.c_int * 8), ("frac", ct.c_int * 8), ("offset", ct.c_int64 * 8),
                ("pred_err", ct.c_double), ("total_bits", ct.c_double), ("pred_bias", ct.c_double),
                ("pred_var_dither", ct.c_double), ("capped", ct.c_int), ("refined", ct.c_int)]


class SolveOpt(ct.Structure):
    _fields_ = [("max_bits", ct.c_int), ("refine", ct.c_int), ("beta", ct.c_double * 8),
                ("margin_gain", ct.c_double * 8), ("margin_src", ct.c_int * 8)]


def lib(threaded=False):
    """The sequential oracle library, or (``threaded``) its OpenMP build for long FP64
    reference rollouts."""
    global _lib, _lib_omp
    if threaded:
        if _lib_omp is None:
            _lib_omp = _bind(ct.CDLL(_build.build(threaded=True)))
        return _lib_omp
    if _lib is None:
        _lib = _bind(ct.CDLL(_build.build()))
    return _lib


def _bind(L):
    P = ct.POINTER
    d, i64, u32 = ct.c_double, ct.c_int64, ct.c_uint32
    L.or_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
    L.or_philox4x32.argtypes = [P(u32), P(u32), ct.c_int, P(u32)]
    L.or_dither_draw.argtypes = [ct.c_uint64, u32, u32, ct.c_int]
    L.or_dither_draw.restype = u32
    L.or_encode.argtypes = [d, ct.c_int, ct.c_int, i64, ct.c_int, u32, P(ct.c_int)]
    L.or_encode.restype = u32
    L.or_decode.argtypes = [u32, ct.c_int, i64]
    L.or_decode.restype = d
    L.or_n_comp.argtypes = [ct.c_int, ct.c_int]
    L.or_layout.argtypes = [ct.c_int, ct.c_int, P(ct.c_int), P(ct.c_int), P(ct.c_int),
                            P(ct.c_int)]
    L.or_pack.argtypes = [ct.c_int, P(ct.c_int), P(ct.c_int), ct.c_int, P(u32), P(u32)]
    L.or_unpack.argtypes = [ct.c_int, P(ct.c_int), P(ct.c_int), P(u32), P(u32)]
    L.or_polar2.argtypes = [P(d), P(d)]
    L.or_polar3.argtypes = [P(d), P(d)]
    L.or_kirchhoff.argtypes = [P(Phys), P(d), P(d)]
    L.or_n_nodes.argtypes = [P(Phys)]
    L.or_p2g.argtypes = [P(Phys), i64, P(d), P(d)]
    L.or_p2g.restype = i64
    L.or_grid_update.argtypes = [P(Phys), P(d)]
    L.or_g2p.argtypes = [P(Phys), i64, P(d), P(d)]
    L.or_g2p.restype = i64
    L.or_step_fp64.argtypes = [P(Phys), i64, P(d), P(d)]
    L.or_step_fp64.restype = i64
    L.or_add_noise.argtypes = [ct.c_int, ct.c_int, i64, P(d), u32, ct.c_uint64, P(d), d]
    L.or_add_noise_matched.argtypes = [ct.c_int, ct.c_int, i64, P(d), u32, ct.c_uint64, P(d), d, ct.c_int]
    L.or_encode_state.argtypes = [P(Codec), i64, P(d), u32, P(u32), P(i64)]
    L.or_decode_state.argtypes = [P(Codec), i64, P(u32), P(d)]
    L.or_step_quant.argtypes = [P(Phys), P(Codec), i64, P(u32), u32, P(d), P(d), P(i64)]
    L.or_tile_keys.argtypes = [P(Phys), i64, P(d), P(i64)]
    L.or_stable_sort.argtypes = [i64, P(i64), i64, P(i64)]
    L.or_n_keys.argtypes = [P(Phys)]
    L.or_n_keys.restype = i64
    L.or_mean_sq_pos.argtypes = [ct.c_int, ct.c_int, i64, P(d)]
    L.or_mean_sq_pos.restype = d
    L.or_scheme_solve.argtypes = [P(SolveIn), P(SolveOut)]
    L.or_scheme_bruteforce.argtypes = [P(SolveIn), ct.c_int, ct.c_int, P(SolveOut)]
    L.or_scheme_options.argtypes = [P(SolveIn), P(SolveOpt), P(SolveOut)]
    if hasattr(L, "or_adjoint_step"):
        _bind_adjoint(L)
    return L


def _bind_adjoint(L):
    P = ct.POINTER
    d, i64 = ct.c_double, ct.c_int64
    L.or_adjoint_step.argtypes = [P(Phys), i64, P(d), P(d), P(d)]


def _p(a, ctype):
    return a.ctypes.data_as(ct.POINTER(ctype))


# ------------------------------------------------------------------------------ codec
DITHER_ROUNDS = 7


def philox(ctr, key, rounds=10):
    """Philox4x32 with `rounds` rounds (10: the published known answers; the dither draws
    use DITHER_ROUNDS)."""
    c = (ct.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ct.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ct.c_uint32 * 4)()
    if rounds == 10:
        lib().or_philox4x32_10(c, k, o)
    else:
        lib().or_philox4x32(c, k, int(rounds), o)
    return [int(v) for v in o]


def dither_draw(seed, slot, step, comp):
    return int(lib().or_dither_draw(seed, slot, step, comp))


def encode(v, bits, frac, offset, dither=False, r=0):
    fl = ct.c_int(0)
    u = lib().or_encode(float(v), bits, frac, int(offset), int(bool(dither)), int(r), ct.byref(fl))
    return int(u), int(fl.value)


def decode(u, frac, offset):
    return float(lib().or_decode(int(u), frac, int(offset)))


def n_comp(dim, material):
    return int(lib().or_n_comp(dim, MATERIALS.get(material, material)))


def comp_fields(dim, material):
    nc = n_comp(dim, material)
    out = []
    for c in range(nc):
        out.append(0 if c < dim else 1 if c < 2 * dim else 2 if c < 2 * dim + dim * dim else 3)
    return out


def layout(dim, material, bits, container=(0, 0, 0, 0)):
    nc = n_comp(dim, material)
    b = (ct.c_int * MAX_COMP)(*bits)
    cont = (ct.c_int * 4)(*container)
    pos = (ct.c_int * MAX_COMP)()
    nw = ct.c_int(0)
    rc = lib().or_layout(dim, MATERIALS.get(material, material), b, cont, pos, ct.byref(nw))
    if rc != 0:
        raise ValueError("layout rejected")
    return [int(pos[c]) for c in range(nc)], int(nw.value)


def pack(bits, bitpos, n_words, u):
    nc = len(bits)
    b = (ct.c_int * MAX_COMP)(*bits)
    p = (ct.c_int * MAX_COMP)(*bitpos)
    uu = (ct.c_uint32 * MAX_COMP)(*[int(x) for x in u])
    w = (ct.c_uint32 * max(n_words, 1))()
    lib().or_pack(nc, b, p, n_words, uu, w)
    return [int(w[i]) for i in range(n_words)]


def unpack(bits, bitpos, words):
    nc = len(bits)
    b = (ct.c_int * MAX_COMP)(*bits)
    p = (ct.c_int * MAX_COMP)(*bitpos)
    w = (ct.c_uint32 * (len(words) + 1))(*[int(x) for x in words])
    uu = (ct.c_uint32 * MAX_COMP)()
    lib().or_unpack(nc, b, p, w, uu)
    return [int(uu[c]) for c in range(nc)]


# ------------------------------------------------------------------------------ scenes
def make_phys(scene):
    ph = Phys()
    ph.dim = scene["dim"]
    ph.material = MATERIALS[scene["material"]]
    ph.grid_log2 = scene["grid_log2"]
    ph.bound = scene.get("bound", 3)
    ph.dt = scene["dt"]
    ph.E = scene.get("E", 0.0)
    ph.nu = scene.get("nu", 0.0)
    ph.bulk = scene.get("bulk", 0.0)
    ph.p_vol = scene["p_vol"]
    ph.p_mass = scene["p_vol"] * scene.get("rho", 1.0)
    g = list(scene.get("gravity", (0.0, -9.8, 0.0))) + [0.0, 0.0, 0.0]
    for a in range(3):
        ph.gravity[a] = g[a]
    return ph


def make_codec(scene, scheme):
    """Expand a per-field scheme {"x": {bits, frac, offset, container}, ...} into the
    per-component codec.  Field order is x, v, C, then F (or J)."""
    dim, mat = scene["dim"], scene["material"]
    nc = n_comp(dim, mat)
    fields = comp_fields(dim, mat)
    names = ["x", "v", "C", "J" if mat == "fluid" else "F"]
    bits = [scheme[names[h]]["bits"] for h in fields]
    container = [scheme[names[h]].get("container", 0) for h in range(4)]
    pos, nw = layout(dim, mat, bits, container)
    cd = Codec()
    cd.n_comp = nc
    cd.n_words = nw
    for c in range(nc):
        f = scheme[names[fields[c]]]
        cd.bits[c] = f["bits"]
        cd.frac[c] = f["frac"]
        cd.offset[c] = int(f["offset"])
        cd.bitpos[c] = pos[c]
        cd.field[c] = fields[c]
    cd.seed = int(scene.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    cd.dither = int(bool(scene.get("dither", True)))
    return cd


def n_nodes(ph):
    return int(lib().or_n_nodes(ct.byref(ph)))


def kirchhoff(ph, FJ):
    FJ = np.ascontiguousarray(FJ, dtype=np.float64).ravel()
    tau = np.zeros(9)
    lib().or_kirchhoff(ct.byref(ph), _p(FJ, ct.c_double), _p(tau, ct.c_double))
    return tau[: ph.dim * ph.dim].reshape(ph.dim, ph.dim)


def polar(F):
    F = np.ascontiguousarray(F, dtype=np.float64)
    R = np.zeros_like(F)
    if F.shape == (2, 2):
        lib().or_polar2(_p(F, ct.c_double), _p(R, ct.c_double))
    else:
        lib().or_polar3(_p(F, ct.c_double), _p(R, ct.c_double))
    return R


def p2g(ph, s):
    s = np.ascontiguousarray(s, dtype=np.float64)
    grid = np.zeros(n_nodes(ph) * (1 + ph.dim))
    oog = lib().or_p2g(ct.byref(ph), s.shape[0], _p(s, ct.c_double), _p(grid, ct.c_double))
    return grid.reshape(-1, 1 + ph.dim), int(oog)


def grid_update(ph, grid):
    g = np.ascontiguousarray(grid, dtype=np.float64).copy()
    lib().or_grid_update(ct.byref(ph), _p(g, ct.c_double))
    return g


def g2p(ph, grid, s):
    g = np.ascontiguousarray(grid, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64).copy()
    lib().or_g2p(ct.byref(ph), s.shape[0], _p(g, ct.c_double), _p(s, ct.c_double))
    return s


def step_fp64(ph, s, grid=None):
    s = np.ascontiguousarray(s, dtype=np.float64).copy()
    if grid is None:
        grid = np.zeros(n_nodes(ph) * (1 + ph.dim))
    lib().or_step_fp64(ct.byref(ph), s.shape[0], _p(s, ct.c_double), _p(grid, ct.c_double))
    return s


def add_noise(dim, material, s, step, seed, sigma, sign, matched=False):
    """s + sign * sigma[field] * xi at every component (the explicit store error of the
    noise-injection estimate; xi uniform with unit variance from the Philox counter
    (particle, step, comp / 4, 0xA5)).  Returns a new array."""
    s = np.ascontiguousarray(s, dtype=np.float64).copy()
    mat = MATERIALS[material] if isinstance(material, str) else int(material)
    if s.ndim != 2 or s.shape[1] != int(lib().or_n_comp(int(dim), mat)):
        raise ValueError("state must be [N, n_comp(dim, material)]")
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    if sg.shape != (4,):
        raise ValueError("sigma holds one value per field")
    lib().or_add_noise_matched(int(dim), mat, s.shape[0], _p(s, ct.c_double), int(step),
                               int(seed) & 0xFFFFFFFFFFFFFFFF, _p(sg, ct.c_double), float(sign), int(bool(matched)))
    return s


def noise_rollout_state(scene, s0, T, sigma, seed, sign, matched=False):
    """The state after T FP64 steps (no re-ordering) from s0 with the explicit error of
    (seed, sign) added after every step (sign 0: none)."""
    ph = make_phys(scene)
    s = np.ascontiguousarray(s0, dtype=np.float64).copy()
    grid = np.zeros(n_nodes(ph) * (1 + ph.dim))
    for t in range(T):
        s = step_fp64(ph, s, grid)
        if sign != 0.0:
            s = add_noise(ph.dim, ph.material, s, t + 1, seed, sigma, sign, matched)
    return s


def noise_rollout_z(scene, s0, T, sigma, seed, sign, measure="mean_sq_pos", matched=False):
    """z of noise_rollout_state."""
    ph = make_phys(scene)
    s = noise_rollout_state(scene, s0, T, sigma, seed, sign, matched)
    if measure == "kinetic_energy":
        return kinetic_energy(ph, s)
    return mean_sq_pos(ph.dim, s)


def encode_state(cd, s, step, stats=None, threaded=False):
    s = np.ascontiguousarray(s, dtype=np.float64)
    N = s.shape[0]
    w = np.zeros((N, cd.n_words), dtype=np.uint32)
    st = stats if stats is not None else np.zeros(N_STATS, dtype=np.int64)
    lib(threaded).or_encode_state(ct.byref(cd), N, _p(s, ct.c_double), step, _p(w, ct.c_uint32),
                                  _p(st, ct.c_int64))
    return w


def decode_state(cd, words, threaded=False):
    words = np.ascontiguousarray(words, dtype=np.uint32)
    N = words.shape[0]
    s = np.zeros((N, cd.n_comp))
    lib(threaded).or_decode_state(ct.byref(cd), N, _p(words, ct.c_uint32), _p(s, ct.c_double))
    return s


def tile_keys(ph, s, threaded=False):
    s = np.ascontiguousarray(s, dtype=np.float64)
    k = np.zeros(s.shape[0], dtype=np.int64)
    lib(threaded).or_tile_keys(ct.byref(ph), s.shape[0], _p(s, ct.c_double), _p(k, ct.c_int64))
    return k


def n_keys(ph):
    return int(lib().or_n_keys(ct.byref(ph)))


def stable_sort(keys, nkeys):
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    perm = np.zeros(keys.shape[0], dtype=np.int64)
    lib().or_stable_sort(keys.shape[0], _p(keys, ct.c_int64), nkeys, _p(perm, ct.c_int64))
    return perm


def mean_sq_pos(dim, s):
    s = np.ascontiguousarray(s, dtype=np.float64)
    return float(lib().or_mean_sq_pos(dim, s.shape[1], s.shape[0], _p(s, ct.c_double)))


class QuantRollout:
    """Oracle rollout of the quantized simulation (Eq. 1) with the same slot ordering as
    the device path: encode at step 0, stable re-sort by tile key at step 0 and after
    every ``resort_every``-th step."""

    def __init__(self, scene, scheme, s0, threaded=False):
        self.threaded = threaded
        self.ph = make_phys(scene)
        self.cd = make_codec(scene, scheme)
        self.resort_every = int(scene.get("resort_every", 8))
        s0 = np.ascontiguousarray(s0, dtype=np.float64)
        self.N = s0.shape[0]
        self.stats = np.zeros(N_STATS, dtype=np.int64)
        self.words = encode_state(self.cd, s0, 0, self.stats, threaded)
        self.ids = np.arange(self.N, dtype=np.int64)
        self.t = 0
        self.grid = np.zeros(n_nodes(self.ph) * (1 + self.ph.dim))
        self.s = np.zeros((self.N, self.cd.n_comp))
        self.resort()

    def resort(self):
        s = decode_state(self.cd, self.words, self.threaded)
        perm = stable_sort(tile_keys(self.ph, s, self.threaded), n_keys(self.ph))
        self.words = np.ascontiguousarray(self.words[perm])
        self.ids = self.ids[perm]

    def step(self, n=1):
        for _ in range(n):
            self.t += 1
            lib(self.threaded).or_step_quant(ct.byref(self.ph), ct.byref(self.cd), self.N,
                                _p(self.words, ct.c_uint32), self.t, _p(self.s, ct.c_double),
                                _p(self.grid, ct.c_double), _p(self.stats, ct.c_int64))
            if self.resort_every > 0 and self.t % self.resort_every == 0:
                self.resort()

    def state(self):
        return decode_state(self.cd, self.words, self.threaded)


class Fp64Rollout:
    """Oracle rollout of the unquantized FP64 simulation, with the same ordering."""

    def __init__(self, scene, s0, threaded=False):
        self.threaded = threaded
        self.ph = make_phys(scene)
        self.resort_every = int(scene.get("resort_every", 8))
        self.s = np.ascontiguousarray(s0, dtype=np.float64).copy()
        self.N = self.s.shape[0]
        self.ids = np.arange(self.N, dtype=np.int64)
        self.grid = np.zeros(n_nodes(self.ph) * (1 + self.ph.dim))
        self.t = 0
        self.resort()

    def resort(self):
        perm = stable_sort(tile_keys(self.ph, self.s, self.threaded), n_keys(self.ph))
        self.s = np.ascontiguousarray(self.s[perm])
        self.ids = self.ids[perm]

    def step(self, n=1):
        for _ in range(n):
            self.t += 1
            lib(self.threaded).or_step_fp64(ct.byref(self.ph), self.N, _p(self.s, ct.c_double),
                                            _p(self.grid, ct.c_double))
            if self.resort_every > 0 and self.t % self.resort_every == 0:
                self.resort()


# ------------------------------------------------------------------------------ adjoint
def adjoint_step(ph, s, sbn):
    """Adjoint of state s_t from the adjoint of s_{t+1} (Sec. 6, Eq. 13)."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    sbn = np.ascontiguousarray(sbn, dtype=np.float64)
    sb = np.zeros_like(s)
    lib().or_adjoint_step(ct.byref(ph), s.shape[0], _p(s, ct.c_double), _p(sbn, ct.c_double),
                          _p(sb, ct.c_double))
    return sb


def mean_sq_pos_seed(dim, s):
    """dz/ds for z = (1/N) sum |x|^2."""
    g = np.zeros_like(s)
    g[:, :dim] = 2.0 * s[:, :dim] / s.shape[0]
    return g


def kinetic_energy(ph, s):
    """z = (1/2) m sum |v|^2 (the kinetic energy used as evaluation function in Sec. 8.1)."""
    d = ph.dim
    return 0.5 * ph.p_mass * float((s[:, d:2 * d] ** 2).sum())


def kinetic_energy_seed(ph, s):
    g = np.zeros_like(s)
    g[:, ph.dim:2 * ph.dim] = ph.p_mass * s[:, ph.dim:2 * ph.dim]
    return g


def rollout_fp64(ph, s0, T):
    """States s_0 .. s_T of the FP64 step (no re-ordering)."""
    states = [np.ascontiguousarray(s0, dtype=np.float64).copy()]
    for _ in range(T):
        states.append(step_fp64(ph, states[-1]))
    return states


def rollout_adjoint(ph, s0, T, seed_fn=None):
    """Reverse mode over a T-step FP64 rollout: returns z, the adjoints dz/ds_t for
    t = 0..T, and g_h = sum_t sum_i (dz/ds_t[h, i])^2 per field (Eq. 8)."""
    dim = ph.dim
    states = rollout_fp64(ph, s0, T)
    if seed_fn == "kinetic":
        z = kinetic_energy(ph, states[-1])
        sb = kinetic_energy_seed(ph, states[-1])
    else:
        z = mean_sq_pos(dim, states[-1])
        sb = seed_fn(states[-1]) if seed_fn else mean_sq_pos_seed(dim, states[-1])
    adj = [None] * (T + 1)
    adj[T] = sb
    for t in range(T - 1, -1, -1):
        adj[t] = adjoint_step(ph, states[t], adj[t + 1])
    nc = states[0].shape[1]
    fields = comp_fields(dim, {0: "neohookean", 1: "corotated", 2: "fluid"}[ph.material])
    g = np.zeros(4)
    for a in adj:
        sq = (a * a).sum(axis=0)
        for c in range(nc):
            g[fields[c]] += sq[c]
    return z, adj, g


# ------------------------------------------------------------------------------ solve
def _solve_in(P, g, lo, hi, z, eps, mode, rounding, kappa):
    si = SolveIn()
    si.H = len(P)
    for h in range(len(P)):
        si.P[h] = P[h]
        si.g[h] = g[h]
        si.lo[h] = lo[h]
        si.hi[h] = hi[h]
    si.kappa = kappa
    si.z = z
    si.eps = eps
    si.mode = 0 if mode == "error" else 1
    si.rounding = 0 if rounding == "paper" else 1
    return si


def _solve_out(so, H):
    return {
        "delta_cont": [so.delta_cont[h] for h in range(H)],
        "bits_paper": [so.bits_paper[h] for h in range(H)],
        "bits": [so.bits[h] for h in range(H)],
        "frac": [so.frac[h] for h in range(H)],
        "offset": [int(so.offset[h]) for h in range(H)],
        "pred_err": so.pred_err,
        "total_bits": so.total_bits,
        "pred_bias": so.pred_bias,
        "pred_var_dither": so.pred_var_dither,
        "capped_mask": so.capped,
        "refined": so.refined,
    }


def scheme_solve(P, g, lo, hi, z, eps, mode="error", rounding="paper", kappa=2.0, max_bits=0, beta=None,
                 margins=None):
    """The solve, then (when given) its options: max_bits, the second-order refinement with
    beta, and window margins {h: (src, gain)}."""
    si = _solve_in(P, g, lo, hi, z, eps, mode, rounding, kappa)
    so = SolveOut()
    rc = lib().or_scheme_solve(ct.byref(si), ct.byref(so))
    if rc != 0:
        raise ValueError(f"oracle scheme solve failed ({rc})")
    op = SolveOpt()
    op.max_bits = int(max_bits)
    if beta is not None:
        op.refine = 1
        for h, b in enumerate(beta):
            op.beta[h] = float(b)
    for h, (src, gain) in (margins or {}).items():
        op.margin_src[h], op.margin_gain[h] = int(src), float(gain)
    rc = lib().or_scheme_options(ct.byref(si), ct.byref(op), ct.byref(so))
    if rc != 0:
        raise ValueError(f"oracle scheme options failed ({rc})")
    return _solve_out(so, len(P))


def scheme_bruteforce(P, g, lo, hi, z, eps, mode="error", kappa=2.0, frac_lo=-8, frac_hi=40):
    si = _solve_in(P, g, lo, hi, z, eps, mode, "exact", kappa)
    so = SolveOut()
    rc = lib().or_scheme_bruteforce(ct.byref(si), frac_lo, frac_hi, ct.byref(so))
    if rc != 0:
        raise ValueError(f"oracle brute force failed ({rc})")
    return _solve_out(so, len(P))


# ------------------------------------------------------------------------------ smoke
class Smoke(ct.Structure):
    _fields_ = [("n", ct.c_int), ("jacobi", ct.c_int), ("dt", ct.c_double), ("buoyancy", ct.c_double),
                ("v_in", ct.c_double), ("src", ct.c_double * 4), ("seed", ct.c_uint64), ("dither", ct.c_int)]


class SmokeScheme(ct.Structure):
    _fields_ = [("bits", ct.c_int * 2), ("frac", ct.c_int * 2), ("offset", ct.c_int64 * 2)]


def _bind_smoke(L):
    P = ct.POINTER
    d = ct.c_double
    L.or_smoke_step.argtypes = [P(Smoke), P(SmokeScheme), ct.c_uint32, P(d), P(d), P(d), P(d)]
    L.or_smoke_step.restype = ct.c_int64
    L.or_smoke_measure.argtypes = [P(Smoke), P(d)]
    L.or_smoke_measure.restype = d
    L.or_smoke_inject.argtypes = [ct.c_int, ct.c_int, ct.c_uint32, ct.c_uint32, d]
    L.or_smoke_noise.argtypes = [ct.c_int, d, d, ct.c_uint64, d]
    L.or_smoke_record.argtypes = [P(ct.c_uint32), ct.c_int64]
    L.or_smoke_record_values.argtypes = [P(ct.c_uint32), P(d), ct.c_int64]
    L.or_smoke_stage.argtypes = [P(Smoke), P(SmokeScheme), ct.c_int, ct.c_int, ct.c_uint32] + [P(d)] * 11
    L.or_smoke_stage.restype = ct.c_int
    L.or_smoke_recorded.restype = ct.c_int64


def _smoke_lib():
    L = lib()
    if not hasattr(L, "_smoke_bound"):
        _bind_smoke(L)
        L._smoke_bound = True
    return L


def make_smoke(scene):
    sm = Smoke()
    sm.n = int(scene["n"])
    sm.jacobi = int(scene.get("jacobi", 64))
    sm.dt = float(scene["dt"])
    sm.buoyancy = float(scene.get("buoyancy", 0.0))
    sm.v_in = float(scene.get("v_in", 0.0))
    for k, x in enumerate(scene.get("src", (0.0, 0.0, -1.0, -1.0))):
        sm.src[k] = float(x)
    sm.seed = int(scene.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    sm.dither = int(bool(scene.get("dither", True)))
    return sm


def make_smoke_scheme(scheme):
    if scheme is None:
        return None
    sc = SmokeScheme()
    for h, name in enumerate(("v", "p")):
        sc.bits[h] = int(scheme[name]["bits"])
        sc.frac[h] = int(scheme[name]["frac"])
        sc.offset[h] = int(scheme[name]["offset"])
    return sc


class SmokeRollout:
    """Oracle rollout of the 2D advection-reflection smoke (unquantized if scheme is None).
    Fields: u [n][n+1] (x-faces), v [n+1][n] (y-faces), d and q [n][n], row = y index."""

    def __init__(self, scene, scheme=None, u0=None, v0=None, d0=None):
        _smoke_lib()
        self.sm = make_smoke(scene)
        self.sch = make_smoke_scheme(scheme)
        n = self.sm.n
        self.u = np.zeros((n, n + 1)) if u0 is None else np.array(u0, dtype=np.float64)
        self.v = np.zeros((n + 1, n)) if v0 is None else np.array(v0, dtype=np.float64)
        self.d = np.zeros((n, n)) if d0 is None else np.array(d0, dtype=np.float64)
        self.q = np.zeros((n, n))
        self.t = 0
        self.saturations = 0

    def step(self, k=1):
        L = lib()
        for _ in range(k):
            self.t += 1
            self.saturations += L.or_smoke_step(ct.byref(self.sm), ct.byref(self.sch) if self.sch is not None else None,
                                                self.t, _p(self.u, ct.c_double), _p(self.v, ct.c_double),
                                                _p(self.d, ct.c_double), _p(self.q, ct.c_double))

    def measure(self):
        return float((self.d ** 2).sum())


def smoke_inject(active, field=0, idx=0, counter=0, delta=0.0):
    _smoke_lib().or_smoke_inject(int(active), int(field), int(idx), int(counter), float(delta))


class smoke_noise:
    """Context: every store of type h (but the reflection and the wall faces) gets
    sign * sigma_h * (+-1), the signs drawn from Philox with key = seed."""

    def __init__(self, sigma, seed, sign):
        self.args = (float(sigma[0]), float(sigma[1]), int(seed) & 0xFFFFFFFFFFFFFFFF, float(sign))

    def __enter__(self):
        _smoke_lib().or_smoke_noise(1, *self.args)
        return self

    def __exit__(self, *exc):
        _smoke_lib().or_smoke_noise(0, 0.0, 0.0, 0, 0.0)
        return False


SMOKE_STAGES = {"advect1": 0, "jacobi": 1, "gradsub2": 2, "advect4": 3, "gradsub5": 4}


def smoke_stage(scene, scheme, stage, step, arg=0, a=None, b=None, q=None, div=None):
    """One stage of the quantized smoke step from given inputs (or_smoke_stage): a, b are
    (u [n][n+1], v [n+1][n]) pairs, q and div [n][n].  Returns the codes every store of the
    stage wrote (in order), the values they were offered (FP64) and the stage's outputs."""
    L = _smoke_lib()
    sm, sch = make_smoke(scene), make_smoke_scheme(scheme)
    n = sm.n

    def arr(x, shape):
        return None if x is None else np.ascontiguousarray(x, dtype=np.float64).reshape(shape)

    au, av = (arr(a[0], (n, n + 1)), arr(a[1], (n + 1, n))) if a is not None else (None, None)
    bu, bv = (arr(b[0], (n, n + 1)), arr(b[1], (n + 1, n))) if b is not None else (None, None)
    qq, dv = arr(q, (n, n)), arr(div, (n, n))
    out = {k: np.zeros(sh) for k, sh in (("u", (n, n + 1)), ("v", (n + 1, n)), ("u2", (n, n + 1)), ("v2", (n + 1, n)),
                                           ("q", (n, n)))}
    cap = 4 * (n + 1) * n + n * n
    codes = np.zeros(cap, dtype=np.uint32)
    xs = np.zeros(cap)
    L.or_smoke_record_values(_p(codes, ct.c_uint32), _p(xs, ct.c_double), cap)

    def ptr(x):
        return None if x is None else _p(x, ct.c_double)

    try:
        rc = L.or_smoke_stage(ct.byref(sm), ct.byref(sch), SMOKE_STAGES[stage], int(arg), int(step), ptr(au), ptr(av),
                              ptr(bu), ptr(bv), ptr(qq), ptr(dv), ptr(out["u"]), ptr(out["v"]), ptr(out["u2"]),
                              ptr(out["v2"]), ptr(out["q"]))
        m = int(L.or_smoke_recorded())
    finally:
        L.or_smoke_record(None, 0)
    if rc != 0:
        raise ValueError(f"oracle smoke stage failed ({rc})")
    return {"codes": codes[:m], "x": xs[:m], **out}


def smoke_store_events(n, jacobi, T):
    """Every quantized store of a T-step run: (type h, field, sample index, store counter)
    with h = 0 velocity, 1 pressure; the order of the step's stores is velocity, jacobi
    pressure iterates, velocity x 3, jacobi pressure iterates, velocity."""
    ev = []
    for t in range(1, T + 1):
        c = 1024 * t
        seq = ["v"] + ["p"] * jacobi + ["v", "v", "v"] + ["p"] * jacobi + ["v"]
        for kind in seq:
            c += 1
            if kind == "v":
                ev += [(0, 0, i, c) for i in range((n + 1) * n)] + [(0, 1, i, c) for i in range(n * (n + 1))]
            else:
                ev += [(1, 2, i, c) for i in range(n * n)]
    return ev


def smoke_codes(scene, scheme, T, u0=None, v0=None, d0=None):
    """The quantized oracle's own code at every store of a T-step run, in store order."""
    L = _smoke_lib()
    n, J = int(scene["n"]), int(scene.get("jacobi", 64))
    size = T * (5 * 2 * n * (n + 1) + 2 * J * n * n)
    buf = np.zeros(size, dtype=np.uint32)
    L.or_smoke_record(_p(buf, ct.c_uint32), size)
    try:
        r = SmokeRollout(scene, scheme, u0, v0, d0)
        r.step(T)
        assert L.or_smoke_recorded() == size
    finally:
        L.or_smoke_record(None, 0)
    return buf
