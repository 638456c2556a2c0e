"""Binding of the quantized 2D Eulerian smoke (``include/qmpm_smoke.h``) and the scheme
workflow of the paper's second error-bounded experiment (Sec. 8.1) on top of it.

Argument marshalling only: every step runs in libqmpm's CUDA kernels (there is no CPU
fallback).  ``Smoke`` wraps a batch handle; ``sensitivities`` estimates Eq. 8's g_h for the
two quantized types (velocity, pressure) by antithetic noise injection in FP32 runs, and
``solve`` hands them with the recorded ranges to the library's Algorithm 1 solve.

Array layouts (row = y index): u [n][n+1] x-faces, v [n+1][n] y-faces, d and q [n][n].
"""
import ctypes as ct

import numpy as np

from . import qmpm
from .qmpm import _check, _dptr, lib

TYPES = ("v", "p")
RANGES = 1  # QMPM_SMOKE_RANGES
PROFILE = 2  # QMPM_SMOKE_PROFILE


def make_config(scene):
    c = qmpm.qmpm_smoke_config_t()
    c.n = int(scene["n"])
    c.jacobi = int(scene.get("jacobi", 64))
    c.dt = float(scene["dt"])
    c.buoyancy = float(scene.get("buoyancy", 0.0))
    c.v_in = float(scene.get("v_in", 0.0))
    for k, x in enumerate(scene.get("src", (1.0, 1.0, -1.0, -1.0))):
        c.src[k] = float(x)
    c.dither = int(bool(scene.get("dither", True)))
    c.flags = (RANGES if scene.get("ranges", False) else 0) | (PROFILE if scene.get("profile", False) else 0)
    return c


def make_scheme(scheme):
    if scheme is None:
        return None
    s = qmpm.qmpm_smoke_scheme_t()
    for h, name in enumerate(TYPES):
        s.bits[h] = int(scheme[name]["bits"])
        s.frac[h] = int(scheme[name]["frac"])
        s.offset[h] = int(scheme[name]["offset"])
    return s


def _f32(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float32)
    assert a.shape == shape, (a.shape, shape)
    return a


class Smoke:
    """A batch of n_scenes smoke scenes sharing one configuration and scheme (None: FP32)."""

    def __init__(self, scene, scheme=None, n_scenes=1, seeds=None, stream=0):
        self.scene = dict(scene)
        self.n = int(scene["n"])
        self.S = int(n_scenes)
        self.quantized = scheme is not None
        self.h = ct.c_void_p()
        cfg = make_config(scene)
        sch = make_scheme(scheme)
        sd = None
        if seeds is not None:
            sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
            assert sd.size == self.S
        _check(lib().qmpm_smoke_create(ct.byref(cfg), ct.byref(sch) if sch is not None else None, self.S,
                                       _dptr(sd, ct.c_uint64) if sd is not None else None, ct.c_void_p(stream),
                                       ct.byref(self.h)))

    def set_state(self, u=None, v=None, d=None, scene=-1):
        n = self.n
        u, v, d = _f32(u, (n, n + 1)), _f32(v, (n + 1, n)), _f32(d, (n, n))
        p = lambda a: _dptr(a, ct.c_float) if a is not None else None  # noqa: E731
        _check(lib().qmpm_smoke_set_state(self.h, int(scene), p(u), p(v), p(d)))

    def _host_ptr(self, a, shape, out=False):
        """Pointer of a host array of every scene (a CPU torch tensor, pinned or not, or a
        numpy array), checked for shape and float32."""
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            assert tuple(a.shape) == shape and str(a.dtype) == "torch.float32" and a.is_contiguous()
            assert a.device.type == "cpu"
            return ct.c_void_p(a.data_ptr())
        assert a.shape == shape and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
        return ct.c_void_p(a.ctypes.data)

    def set_states(self, u=None, v=None, d=None):
        """Every scene's state from host arrays u [S][n][n+1], v [S][n+1][n], d [S][n][n]."""
        n, S = self.n, self.S
        _check(lib().qmpm_smoke_set_states(self.h, self._host_ptr(u, (S, n, n + 1)), self._host_ptr(v, (S, n + 1, n)),
                                           self._host_ptr(d, (S, n, n))))

    def get_states(self, u=None, v=None, d=None):
        """Every scene's decoded state into host arrays shaped as in set_states."""
        n, S = self.n, self.S
        _check(lib().qmpm_smoke_get_states(self.h, self._host_ptr(u, (S, n, n + 1)), self._host_ptr(v, (S, n + 1, n)),
                                           self._host_ptr(d, (S, n, n))))

    def set_noise(self, sigma, noise_seeds, signs):
        sg = (ct.c_float * 2)(float(sigma[0]), float(sigma[1]))
        ns = np.ascontiguousarray(np.asarray(noise_seeds, dtype=np.uint64))
        si = np.ascontiguousarray(np.asarray(signs, dtype=np.float32))
        assert ns.size == self.S and si.size == self.S
        _check(lib().qmpm_smoke_set_noise(self.h, sg, _dptr(ns, ct.c_uint64), _dptr(si, ct.c_float)))

    def trace_len(self, steps):
        n, J = self.n, int(self.scene.get("jacobi", 64))
        return steps * (10 * n * (n + 1) + 2 * J * n * n)

    def step(self, steps=1, trace=None):
        """trace: a CUDA int32 tensor of trace_len(steps) elements that receives scene 0's
        store codes (plain launches), or None (CUDA graph replay)."""
        if trace is None:
            _check(lib().qmpm_smoke_step(self.h, int(steps), None, 0))
        else:
            import torch
            # the tensor's allocation and fill are ordered on torch's stream, the handle's
            # kernels on its own: let the former finish first
            torch.cuda.current_stream(trace.device).synchronize()
            _check(lib().qmpm_smoke_step(self.h, int(steps), ct.c_void_p(trace.data_ptr()), int(trace.numel())))

    def measure(self):
        z = np.zeros(self.S)
        _check(lib().qmpm_smoke_measure(self.h, _dptr(z, ct.c_double)))
        return z

    STAGES = {"advect1": 0, "jacobi": 1, "gradsub2": 2, "advect4": 3, "gradsub5": 4}

    def stage(self, stage, step, arg=0, a=None, b=None, q=None, div=None):
        """One stage of a quantized step on scene 0 from given inputs (qmpm_smoke_stage):
        a, b are (u, v) pairs, q and div cell arrays.  Returns the codes of the stage's
        stores in order.  Overwrites the scene's stored fields."""
        n = self.n
        nu = n * (n + 1)
        m = {"jacobi": n * n, "gradsub2": 4 * nu}.get(stage, 2 * nu)
        out = np.zeros(m, dtype=np.uint32)
        au, av = (_f32(a[0], (n, n + 1)), _f32(a[1], (n + 1, n))) if a is not None else (None, None)
        bu, bv = (_f32(b[0], (n, n + 1)), _f32(b[1], (n + 1, n))) if b is not None else (None, None)
        qq, dv = _f32(q, (n, n)), _f32(div, (n, n))
        p = lambda x: _dptr(x, ct.c_float) if x is not None else None  # noqa: E731
        _check(lib().qmpm_smoke_stage(self.h, self.STAGES[stage], int(arg), int(step), p(au), p(av), p(bu), p(bv),
                                      p(qq), p(dv), _dptr(out, ct.c_uint32)))
        return out

    def readback(self, scene=0):
        n = self.n
        out = {"u": np.zeros((n, n + 1), np.float32), "v": np.zeros((n + 1, n), np.float32),
               "d": np.zeros((n, n), np.float32), "q": np.zeros((n, n), np.float32)}
        _check(lib().qmpm_smoke_readback(self.h, int(scene), *[_dptr(out[k], ct.c_float) for k in "uvdq"]))
        return out

    def ranges(self):
        lo = np.zeros((self.S, 2), np.float32)
        hi = np.zeros((self.S, 2), np.float32)
        sat = np.zeros((self.S, 2), np.int64)
        _check(lib().qmpm_smoke_ranges(self.h, _dptr(lo, ct.c_float), _dptr(hi, ct.c_float), _dptr(sat, ct.c_int64)))
        return lo, hi, sat

    def info(self):
        out = qmpm.qmpm_smoke_info_t()
        _check(lib().qmpm_smoke_info(self.h, ct.byref(out)))
        return out.as_dict()

    def profile(self):
        """Device ms of the steps since the last call, of their Jacobi launches, and the
        number of those launches (handles created with scene["profile"] = True)."""
        a, b, k = ct.c_double(), ct.c_double(), ct.c_int64()
        _check(lib().qmpm_smoke_profile(self.h, ct.byref(a), ct.byref(b), ct.byref(k)))
        return {"step_ms": a.value, "jacobi_ms": b.value, "jacobi_launches": k.value}

    def close(self):
        if self.h is not None and self.h.value:
            _check(lib().qmpm_smoke_destroy(self.h))
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def reference(scene, T, state=None):
    """FP32 run of one scene: z, the per-type value ranges of every store, and the state."""
    with Smoke(dict(scene, ranges=True), None, 1) as s:
        if state is not None:
            s.set_state(*state)
        s.step(T)
        z = float(s.measure()[0])
        lo, hi, _ = s.ranges()
        return {"z": z, "lo": lo[0].astype(float), "hi": hi[0].astype(float), "state": s.readback(0)}


def sensitivities(scene, T, pairs=32, sigma=(3e-3, 3e-5), seed=0, state=None, z0=None):
    """Eq. 8's g_h = sum over the stores of type h of (dz/dstore)^2, for h = velocity,
    pressure, by antithetic noise injection: scenes 2k and 2k+1 of a batch get the same
    +-sigma_h noise at every store of type h with opposite signs, and
    E[((z+ - z-) / 2)^2] = sigma_h^2 g_h to second order.  The pairs' means give the
    second-order term as well: E[(z+ + z-) / 2] - z0 = sigma_h^2 beta_h with
    beta_h = (1/2) sum over the stores of d^2 z / dstore^2 (z0: the noise-free run).
    Returns a dict with g, beta, their standard errors, and the per-pair estimates."""
    if z0 is None:
        z0 = reference(scene, T, state)["z"]
    g, se, beta, beta_se, per = np.zeros(2), np.zeros(2), np.zeros(2), np.zeros(2), []
    for h in range(2):
        sg = [0.0, 0.0]
        sg[h] = float(sigma[h])
        S = 2 * pairs
        ns = np.repeat(np.arange(pairs, dtype=np.uint64) + np.uint64(1 + 7919 * seed + 104729 * h), 2)
        signs = np.tile(np.array([1.0, -1.0], np.float32), pairs)
        with Smoke(scene, None, S) as s:
            if state is not None:
                s.set_state(*state)
            s.set_noise(sg, ns, signs)
            s.step(T)
            z = s.measure()
        est = ((z[0::2] - z[1::2]) / 2.0) ** 2 / sg[h] ** 2
        mid = ((z[0::2] + z[1::2]) / 2.0 - z0) / sg[h] ** 2
        g[h], se[h] = est.mean(), est.std(ddof=1) / np.sqrt(pairs)
        beta[h], beta_se[h] = mid.mean(), mid.std(ddof=1) / np.sqrt(pairs)
        per.append(est)
    return {"g": g, "g_se": se, "beta": beta, "beta_se": beta_se, "per_pair": per, "z0": z0,
            "sigma": list(sigma)}


def predicted_moments(frac, g, beta):
    """Predicted bias and variance of z under dithered stores (rounding error of variance
    Delta_h^2 / 6 per store, Sec. 5): bias = sum_h beta_h Delta_h^2 / 6 and
    var = sum_h g_h Delta_h^2 / 6 (Eq. 8's linear term with the dither's variance)."""
    d2 = np.array([2.0 ** (-2 * f) for f in frac])
    return float(np.dot(beta, d2) / 6.0), float(np.dot(g, d2) / 6.0)


def solve_types(P, g, lo, hi, z, eps, kappa=2.0, max_bits=24, beta=None):
    """qmpm_scheme_solve for the smoke's two types (velocity, pressure): Algorithm 1 with
    the ranges widened by kappa, each type held at max_bits, and with beta the solve's
    second-order refinement (fraction bits added, one at a time to the type with the largest
    drop of the predicted bias^2 + variance per stored bit, until bias^2 + var <= (eps z)^2:
    the bound of Eq. 6 on the second moment with the term Eq. 8 leaves out).  Returns the
    scheme dict and the solve report."""
    res = qmpm.qmpm_scheme_solve(P, list(g), list(lo), list(hi), z, eps, kappa=kappa, max_bits=max_bits,
                                 beta=None if beta is None else list(beta))
    scheme = {name: dict(bits=int(res["bits"][h]), frac=int(res["frac"][h]), offset=int(res["offset"][h]))
              for h, name in enumerate(TYPES)}
    return scheme, res


def bias_aware_scheme(scene, T, eps, ref, g, beta, P, pairs=32, iters=3, state=None, max_bits=24, kappa=2.0):
    """The solve's second-order refinement (solve_types with beta), with the second-order
    term re-estimated at the refined scheme's own noise scale (sigma_h = Delta_h / sqrt(6),
    the dither's spread): the shift of z is not quadratic in the noise scale (the advection
    samples piecewise-bilinearly), so the estimate taken at the sensitivity run's scale is
    only a start.  Stops when the scheme repeats; where the last two differ, keeps the finer
    fraction per type.  ref: the FP32 run (z, ranges).  Returns the scheme and the last
    beta."""
    def refined(b):
        return solve_types(P, g, ref["lo"], ref["hi"], ref["z"], eps, kappa=kappa, max_bits=max_bits, beta=b)[0]
    sch = refined(beta)
    prev = None
    for _ in range(iters):
        sig = tuple(2.0 ** -sch[t]["frac"] / 6 ** 0.5 for t in TYPES)
        beta = sensitivities(scene, T, pairs, sig, state=state, z0=ref["z"])["beta"]
        prev, sch = sch, refined(beta)
        if sch == prev:
            break
    if prev is not None and sch != prev:
        sch = {t: (sch[t] if sch[t]["frac"] >= prev[t]["frac"] else prev[t]) for t in TYPES}
    return sch, beta


def solve(scene, T, eps, pairs=32, sigma=(3e-3, 3e-5), kappa=2.0, state=None, max_bits=24, bias_aware=False):
    """Scheme for the error bound eps on z (Algorithm 1 with the recorded ranges widened by
    kappa about their midpoint, Sec. 3.1); bias_aware adds the bits of the solve's
    second-order refinement.  Returns (scheme dict, report)."""
    n = int(scene["n"])
    ref = reference(scene, T, state)
    sens = sensitivities(scene, T, pairs, sigma, state=state, z0=ref["z"])
    g = sens["g"]
    P = [2.0 * n * (n + 1), float(n * n)]
    scheme, res = solve_types(P, g, ref["lo"], ref["hi"], ref["z"], eps, kappa=kappa, max_bits=max_bits)
    capped = [TYPES[h] for h in range(2) if res["capped_mask"] >> h & 1]
    beta = sens["beta"]
    if bias_aware:
        scheme, beta = bias_aware_scheme(scene, T, eps, ref, g, beta, P, pairs, state=state, max_bits=max_bits,
                                         kappa=kappa)
    frac = [scheme[t]["frac"] for t in TYPES]
    bias, var = predicted_moments(frac, g, beta)
    bits_state = P[0] * scheme["v"]["bits"] + 32.0 * n * n
    rep = {"z": ref["z"], "g": list(g), "g_se": list(sens["g_se"]), "beta": list(beta),
           "beta_se": list(sens["beta_se"]), "lo": list(ref["lo"]), "hi": list(ref["hi"]),
           "solve": res, "capped": capped, "P": P, "pred_bias": bias, "pred_sigma": var ** 0.5,
           "compression_state": (P[0] + n * n) * 32.0 / bits_state,
           "compression_quantized": (P[0] + P[1]) * 32.0 / (P[0] * scheme["v"]["bits"] + P[1] * scheme["p"]["bits"])}
    return scheme, rep


def error_bound_protocol(scene, T, eps_list, runs=20, z_ref=None, pairs=32, seed0=1000, variants=(False, True)):
    """The error-bounded experiment of Sec. 8.1 on the smoke: per eps, the scheme Algorithm 1
    solves from the noise-injection sensitivities and the FP32 run's ranges (and, for the
    bias-aware variant, the bits bias_aware_scheme adds), then `runs` quantized runs (one batch,
    dither seeds seed0 + r); success = |z~ - z| <= 3 eps z."""
    n = int(scene["n"])
    ref = reference(scene, T)
    z0 = ref["z"] if z_ref is None else z_ref
    sens = sensitivities(scene, T, pairs, z0=ref["z"])
    g = sens["g"]
    P = [2.0 * n * (n + 1), float(n * n)]
    out = []
    for eps in eps_list:
        paper, res = solve_types(P, g, ref["lo"], ref["hi"], ref["z"], eps, kappa=2.0, max_bits=24)
        for aware in variants:
            beta = sens["beta"]
            scheme = paper
            if aware:
                scheme, beta = bias_aware_scheme(scene, T, eps, ref, g, beta, P, pairs)
            with Smoke(scene, scheme, runs, seeds=[seed0 + r for r in range(runs)]) as s:
                s.step(T)
                zs = s.measure()
                _, _, sat = s.ranges()
            dev = zs - z0
            bits = [scheme["v"]["bits"], scheme["p"]["bits"]]
            frac = [scheme["v"]["frac"], scheme["p"]["frac"]]
            pb, pv = predicted_moments(frac, g, beta)
            out.append({
                "eps": eps, "solve": "bias-aware" if aware else "Algorithm 1", "bits": bits, "frac": frac,
                "bits_paper": [int(b) for b in res["bits_paper"]],
                "pred_sigma": float(np.sqrt(pv / 2.0)), "pred_sigma_dither": float(np.sqrt(pv)),
                "pred_bias": pb, "obs_rms": float(np.sqrt(np.mean(dev ** 2))), "bias": float(dev.mean()),
                "z_ref": z0, "z_mean": float(zs.mean()), "z_std": float(zs.std(ddof=1)) if runs > 1 else 0.0,
                "success_3eps": float(np.mean(np.abs(dev) <= 3 * eps * abs(z0))),
                "success_eps": float(np.mean(np.abs(dev) <= eps * abs(z0))),
                "saturations": int(sat.sum()),
                "compression": 3 * 32.0 / (2 * bits[0] + bits[1]), "runs": runs,
            })
    return {"z_ref": z0, "g": list(g), "g_se": list(sens["g_se"]), "beta": list(sens["beta"]),
            "beta_se": list(sens["beta_se"]), "lo": list(ref["lo"]), "hi": list(ref["hi"]), "results": out}
